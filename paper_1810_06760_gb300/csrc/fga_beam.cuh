// Device functions of one beam: model sampling, the right-hand side of the FGA ODEs and the
// reconstruction record.  Templated on the arithmetic type R (float for the FP32 path, double
// for the FP64 path) and on the medium kind, so that a constant medium compiles without any
// derivative arithmetic.
#pragma once

#include "fga_internal.cuh"

namespace fga {

template <typename R> struct Real;
template <> struct Real<float> {
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    // 1/x for x > 0 as rsqrt(x)^2: two instructions, a few ulp (FP32 only; FP64 divides)
    static __device__ __forceinline__ float rcp_pos_(float x) {
        const float r = rsqrtf(x);
        return r * r;
    }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }
};
template <> struct Real<double> {
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double rcp_pos_(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }
};

// model parameter in the kernel's precision (double field for FP64, its FP32 copy for FP32)
template <typename R> __device__ __forceinline__ R mp(double d, float f);
template <> __device__ __forceinline__ float mp<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double mp<double>(double d, float) { return d; }

// ---------------------------------------------------------------------------------------------
// A0: c, grad c, Hessian c at x (10 fields: c, c1, c2, c3, c11, c12, c13, c22, c23, c33)
// ---------------------------------------------------------------------------------------------
template <typename R, int MED>
__device__ __forceinline__ void model_eval(const ModelDev &M, int wave, const R x[3], R c[10]) {
    if (MED == FGA_MEDIUM_CONST) {
        c[0] = wave ? mp<R>(M.cs0, M.fcs0) : mp<R>(M.cp0, M.fcp0);
#pragma unroll
        for (int f = 1; f < 10; f++) c[f] = R(0);
    } else if (MED == FGA_MEDIUM_SINE) {
        R s[3], k[3];
#pragma unroll
        for (int d = 0; d < 3; d++) Real<R>::sincospi_(R(2) * x[d], &s[d], &k[d]);
        const R A = mp<R>(M.amp, M.famp), w = R(6.283185307179586476925286766559);
        const R sc = wave ? mp<R>(M.cs_ratio, M.fcs_ratio) : R(1);
        const R Aw = A * w * sc, Aww = A * w * w * sc;
        const R s123 = s[0] * s[1] * s[2];
        c[0] = sc * (mp<R>(M.cp0, M.fcp0) + A * s123);
        c[1] = Aw * k[0] * s[1] * s[2];
        c[2] = Aw * s[0] * k[1] * s[2];
        c[3] = Aw * s[0] * s[1] * k[2];
        c[4] = -Aww * s123;
        c[5] = Aww * k[0] * k[1] * s[2];
        c[6] = Aww * k[0] * s[1] * k[2];
        c[7] = -Aww * s123;
        c[8] = Aww * s[0] * k[1] * k[2];
        c[9] = -Aww * s123;
    } else if (MED == FGA_MEDIUM_GRID) {
        const float4 *__restrict__ G = wave ? M.gs : M.gp;
        int i[3];
        R fr[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            R t = (x[d] - mp<R>(M.o[d], M.fo[d])) * mp<R>(M.inv_h[d], M.finv_h[d]);
            const R hi = R(M.n[d] - 1);
            t = t < R(0) ? R(0) : (t > hi ? hi : t);
            int id = (int)Real<R>::floor_(t);
            id = id > M.n[d] - 2 ? M.n[d] - 2 : id;
            i[d] = id;
            fr[d] = t - R(id);
        }
        const int64_t s1 = M.n[2], s0 = (int64_t)M.n[1] * M.n[2];
        const int64_t base = (int64_t)i[0] * s0 + (int64_t)i[1] * s1 + i[2];
        if constexpr (sizeof(R) == 4) {
            // FP32: the 10 fields as 5 pairs, each lerp step one packed FP32x2 FMA
            float2 acc2[5];
#pragma unroll
            for (int f = 0; f < 5; f++) acc2[f] = make_float2(0.f, 0.f);
            const float2 f2 = make_float2(fr[2], fr[2]), m1 = make_float2(-1.f, -1.f);
#pragma unroll
            for (int a = 0; a < 2; a++) {
                float2 e2[5];
#pragma unroll
                for (int f = 0; f < 5; f++) e2[f] = make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < 2; b++) {
                    const int64_t node = base + a * s0 + b * s1;
                    const float4 *p0 = G + 3 * node;
                    const float4 u0 = __ldg(p0), u1 = __ldg(p0 + 1), u2 = __ldg(p0 + 2);
                    const float4 v0 = __ldg(p0 + 3), v1 = __ldg(p0 + 4), v2 = __ldg(p0 + 5);
                    const float2 lo[5] = {make_float2(u0.x, u0.y), make_float2(u0.z, u0.w), make_float2(u1.x, u1.y),
                                          make_float2(u1.z, u1.w), make_float2(u2.x, u2.y)};
                    const float2 hi[5] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                                          make_float2(v1.z, v1.w), make_float2(v2.x, v2.y)};
                    const float wb = b ? fr[1] : 1.0f - fr[1];
                    const float2 wb2 = make_float2(wb, wb);
#pragma unroll
                    for (int f = 0; f < 5; f++) {
                        const float2 d = __ffma2_rn(lo[f], m1, hi[f]);   // hi - lo
                        const float2 t = __ffma2_rn(f2, d, lo[f]);       // lo + fr2 (hi - lo)
                        e2[f] = __ffma2_rn(wb2, t, e2[f]);
                    }
                }
                const float wa = a ? fr[0] : 1.0f - fr[0];
                const float2 wa2 = make_float2(wa, wa);
#pragma unroll
                for (int f = 0; f < 5; f++) acc2[f] = __ffma2_rn(wa2, e2[f], acc2[f]);
            }
#pragma unroll
            for (int f = 0; f < 5; f++) {
                c[2 * f] = acc2[f].x;
                c[2 * f + 1] = acc2[f].y;
            }
        } else {
        R acc[10];
#pragma unroll
        for (int f = 0; f < 10; f++) acc[f] = R(0);
#pragma unroll
        for (int a = 0; a < 2; a++) {
            R e[10];
#pragma unroll
            for (int f = 0; f < 10; f++) e[f] = R(0);
#pragma unroll
            for (int b = 0; b < 2; b++) {
                const int64_t node = base + a * s0 + b * s1;
                const float4 *p0 = G + 3 * node;
                const float4 u0 = __ldg(p0), u1 = __ldg(p0 + 1), u2 = __ldg(p0 + 2);
                const float4 v0 = __ldg(p0 + 3), v1 = __ldg(p0 + 4), v2 = __ldg(p0 + 5);
                const float lo[10] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y};
                const float hi[10] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y};
                const R wb = b ? fr[1] : R(1) - fr[1];
#pragma unroll
                for (int f = 0; f < 10; f++) {
                    const R l = (R)lo[f];
                    e[f] += wb * (l + fr[2] * ((R)hi[f] - l));
                }
            }
            const R wa = a ? fr[0] : R(1) - fr[0];
#pragma unroll
            for (int f = 0; f < 10; f++) acc[f] += wa * e[f];
        }
#pragma unroll
        for (int f = 0; f < 10; f++) c[f] = acc[f];
        }
    } else {  // layered
        int l = 0;
        for (int q = 0; q < M.nlay - 1; q++) l += (x[2] >= mp<R>(M.zif[q], M.fzif[q])) ? 1 : 0;
        c[0] = wave ? mp<R>(M.lcs[l], M.flcs[l]) : mp<R>(M.lcp[l], M.flcp[l]);
#pragma unroll
        for (int f = 1; f < 10; f++) c[f] = R(0);
    }
}

// S polarisation frame: N_sh = e x P / |e x P| (e = e3, or e1 for near-vertical beams),
// N_sv = N_sh x P/|P|.  Returns |e x P| (and its reciprocal in *inv when given).
template <typename R>
__device__ __forceinline__ R s_frame(const R P[3], bool ref_e1, R Nsv[3], R Nsh[3], R *inv = nullptr) {
    R v0, v1, v2;
    if (ref_e1) {
        v0 = R(0);
        v1 = -P[2];
        v2 = P[1];
    } else {
        v0 = -P[1];
        v1 = P[0];
        v2 = R(0);
    }
    const R v2s = v0 * v0 + v1 * v1 + v2 * v2;
    const R iv = Real<R>::rsqrt_(v2s);
    const R vn = v2s * iv;
    if (inv) *inv = iv;
    Nsh[0] = v0 * iv;
    Nsh[1] = v1 * iv;
    Nsh[2] = v2 * iv;
    const R ip = Real<R>::rsqrt_(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    Nsv[0] = (Nsh[1] * P[2] - Nsh[2] * P[1]) * ip;
    Nsv[1] = (Nsh[2] * P[0] - Nsh[0] * P[2]) * ip;
    Nsv[2] = (Nsh[0] * P[1] - Nsh[1] * P[0]) * ip;
    return vn;
}

// A beam state into the frame x' = Rm x (with transpose, x' = Rm^T x), in FP64: P, Q when with_q, and
// each row m of dzQ and dzP (the vectors dQ/dz_m, dP/dz_m) rotate; an S beam's polarisation vector
// a_sv N_sv + a_sh N_sh rotates with it and is re-expressed in the S frame of the rotated P, whose
// reference axis (FL_REF_E1 in fl) follows the decomposition's rule (e1 when |P_h|^2 < 0.01 |P|^2).
template <typename R>
__device__ void rotate_state(const double *Rm, bool transpose, bool with_q, R *y, int &fl) {
    auto rot = [&](const double *v, double *o) {
        for (int i = 0; i < 3; i++)
            o[i] = transpose ? Rm[i] * v[0] + Rm[3 + i] * v[1] + Rm[6 + i] * v[2]
                             : Rm[3 * i] * v[0] + Rm[3 * i + 1] * v[1] + Rm[3 * i + 2] * v[2];
    };
    const double Pold[3] = {(double)y[F_P], (double)y[F_P + 1], (double)y[F_P + 2]};
    double v[3], o[3];
    for (int base : {F_Q, F_P}) {
        if (base == F_Q && !with_q) continue;
        for (int i = 0; i < 3; i++) v[i] = (double)y[base + i];
        rot(v, o);
        for (int i = 0; i < 3; i++) y[base + i] = (R)o[i];
    }
    for (int base : {F_DQ, F_DP})
        for (int m = 0; m < 3; m++)
            for (int part = 0; part < 2; part++) {
                for (int j = 0; j < 3; j++) v[j] = (double)y[base + 2 * (3 * m + j) + part];
                rot(v, o);
                for (int j = 0; j < 3; j++) y[base + 2 * (3 * m + j) + part] = (R)o[j];
            }
    if ((fl & FL_CLASS_MASK) < 2) return;
    double Nsv[3], Nsh[3], Ar[3], Ai[3], Arr[3], Air[3];
    s_frame<double>(Pold, (fl & FL_REF_E1) != 0, Nsv, Nsh);
    for (int i = 0; i < 3; i++) {
        Ar[i] = (double)y[F_A0] * Nsv[i] + (double)y[F_A1] * Nsh[i];
        Ai[i] = (double)y[F_A0 + 1] * Nsv[i] + (double)y[F_A1 + 1] * Nsh[i];
    }
    rot(Ar, Arr);
    rot(Ai, Air);
    double P[3];
    rot(Pold, P);
    const bool r1 = (P[0] * P[0] + P[1] * P[1]) < 0.01 * (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    fl = r1 ? (fl | FL_REF_E1) : (fl & ~FL_REF_E1);
    s_frame<double>(P, r1, Nsv, Nsh);
    y[F_A0] = (R)(Arr[0] * Nsv[0] + Arr[1] * Nsv[1] + Arr[2] * Nsv[2]);
    y[F_A0 + 1] = (R)(Air[0] * Nsv[0] + Air[1] * Nsv[1] + Air[2] * Nsv[2]);
    y[F_A1] = (R)(Arr[0] * Nsh[0] + Arr[1] * Nsh[1] + Arr[2] * Nsh[2]);
    y[F_A1 + 1] = (R)(Air[0] * Nsh[0] + Air[1] * Nsh[1] + Air[2] * Nsh[2]);
}

// complex helpers on (re, im) pairs kept in scalars
template <typename R> struct C2 {
    R r, i;
};
template <typename R> __device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename R> __device__ __forceinline__ C2<R> csub(C2<R> a, C2<R> b) { return {a.r - b.r, a.i - b.i}; }
template <typename R> __device__ __forceinline__ C2<R> cmulsub(C2<R> a, C2<R> b, C2<R> c, C2<R> d) {
    // a*b - c*d
    return {a.r * b.r - a.i * b.i - (c.r * d.r - c.i * d.i), a.r * b.i + a.i * b.r - (c.r * d.i + c.i * d.r)};
}

// ---------------------------------------------------------------------------------------------
// A3: right-hand side of the beam ODEs (Eqs. char_plus/char_minus, DzDt, amp_P, amp_SV, amp_SH)
//   Q' = sg c P^,  P' = -sg |P| grad c
//   dzQ'_mj = sg [ (c/|P|) dzP_mj + (u_m - (c/|P|) v_m) P^_j ],   u = dzQ grad c,  v = dzP P^
//   dzP'_mj = -sg [ |P| (dzQ Hess c)_mj + v_m (grad c)_j ]
//   gamma = sg grad c . P^ + tr(Z^-1 Z')/2,  Z = dzQ + i dzP, via the cofactor matrix of Z
//   P: a' = gamma a;  S: a_sv' = gamma a_sv - a_sh w,  a_sh' = gamma a_sh + a_sv w,
//      w = dN_sh/dt . N_sv = (e x P') . N_sv / |e x P|
// ---------------------------------------------------------------------------------------------
template <typename R, int WAVE, int MED>
__device__ __forceinline__ void beam_rhs(const ModelDev &M, R sg, bool ref_e1, const R *__restrict__ y,
                                         R *__restrict__ f) {
    R cf[10];
    const R Q[3] = {y[F_Q], y[F_Q + 1], y[F_Q + 2]};
    model_eval<R, MED>(M, WAVE, Q, cf);
    const R c = cf[0];
    const R g[3] = {cf[1], cf[2], cf[3]};
    const R H[3][3] = {{cf[4], cf[5], cf[6]}, {cf[5], cf[7], cf[8]}, {cf[6], cf[8], cf[9]}};
    const R P[3] = {y[F_P], y[F_P + 1], y[F_P + 2]};
    const R p2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const R ip = Real<R>::rsqrt_(p2);
    const R pn = p2 * ip;   // |P| without a division
    const R Ph[3] = {P[0] * ip, P[1] * ip, P[2] * ip};
    const R sc = sg * c;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        f[F_Q + d] = sc * Ph[d];
        f[F_P + d] = -sg * pn * g[d];
    }
    const R cip = c * ip;
    if constexpr (sizeof(R) == 4) {
        // FP32: each complex entry (re, im) as one packed FP32x2 value
        auto ld = [&](int off) { return make_float2(y[off], y[off + 1]); };
        auto bc = [](float v) { return make_float2(v, v); };
        const float2 sgcip = bc(sg * cip), msgpn = bc(-sg * pn);
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float2 u = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f);
#pragma unroll
            for (int l = 0; l < 3; l++) {
                u = __ffma2_rn(ld(F_DQ + 2 * (3 * m + l)), bc(g[l]), u);
                v = __ffma2_rn(ld(F_DP + 2 * (3 * m + l)), bc(Ph[l]), v);
            }
            const float2 wv = __ffma2_rn(bc(-cip), v, u);   // u - (c/|P|) v
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const float2 fq = __ffma2_rn(wv, bc(sg * Ph[j]), __fmul2_rn(sgcip, ld(F_DP + 2 * (3 * m + j))));
                f[F_DQ + 2 * (3 * m + j)] = fq.x;
                f[F_DQ + 2 * (3 * m + j) + 1] = fq.y;
                float2 hh = __fmul2_rn(ld(F_DQ + 2 * (3 * m)), bc(H[0][j]));
                hh = __ffma2_rn(ld(F_DQ + 2 * (3 * m + 1)), bc(H[1][j]), hh);
                hh = __ffma2_rn(ld(F_DQ + 2 * (3 * m + 2)), bc(H[2][j]), hh);
                const float2 fp = __ffma2_rn(v, bc(-sg * g[j]), __fmul2_rn(msgpn, hh));
                f[F_DP + 2 * (3 * m + j)] = fp.x;
                f[F_DP + 2 * (3 * m + j) + 1] = fp.y;
            }
        }
    } else {
#pragma unroll
    for (int m = 0; m < 3; m++) {
        R ur = R(0), ui = R(0), vr = R(0), vi = R(0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            ur += y[F_DQ + 2 * (3 * m + l)] * g[l];
            ui += y[F_DQ + 2 * (3 * m + l) + 1] * g[l];
            vr += y[F_DP + 2 * (3 * m + l)] * Ph[l];
            vi += y[F_DP + 2 * (3 * m + l) + 1] * Ph[l];
        }
        const R wr = ur - cip * vr, wi = ui - cip * vi;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            f[F_DQ + 2 * (3 * m + j)] = sg * (cip * y[F_DP + 2 * (3 * m + j)] + wr * Ph[j]);
            f[F_DQ + 2 * (3 * m + j) + 1] = sg * (cip * y[F_DP + 2 * (3 * m + j) + 1] + wi * Ph[j]);
            R hr = R(0), hi = R(0);
#pragma unroll
            for (int l = 0; l < 3; l++) {
                hr += y[F_DQ + 2 * (3 * m + l)] * H[l][j];
                hi += y[F_DQ + 2 * (3 * m + l) + 1] * H[l][j];
            }
            f[F_DP + 2 * (3 * m + j)] = -sg * (pn * hr + vr * g[j]);
            f[F_DP + 2 * (3 * m + j) + 1] = -sg * (pn * hi + vi * g[j]);
        }
    }
    }
    // Z = dzQ + i dzP and Z' likewise
    C2<R> Z[3][3], Zd[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int e = 2 * (3 * m + j);
            Z[m][j] = {y[F_DQ + e] - y[F_DP + e + 1], y[F_DQ + e + 1] + y[F_DP + e]};
            Zd[m][j] = {f[F_DQ + e] - f[F_DP + e + 1], f[F_DQ + e + 1] + f[F_DP + e]};
        }
    // cofactors C_ij; tr(Z^-1 Z') = sum_ij C_ij Z'_ij / det Z
    C2<R> Cf[3][3];
    Cf[0][0] = cmulsub(Z[1][1], Z[2][2], Z[1][2], Z[2][1]);
    Cf[0][1] = cmulsub(Z[1][2], Z[2][0], Z[1][0], Z[2][2]);
    Cf[0][2] = cmulsub(Z[1][0], Z[2][1], Z[1][1], Z[2][0]);
    Cf[1][0] = cmulsub(Z[0][2], Z[2][1], Z[0][1], Z[2][2]);
    Cf[1][1] = cmulsub(Z[0][0], Z[2][2], Z[0][2], Z[2][0]);
    Cf[1][2] = cmulsub(Z[0][1], Z[2][0], Z[0][0], Z[2][1]);
    Cf[2][0] = cmulsub(Z[0][1], Z[1][2], Z[0][2], Z[1][1]);
    Cf[2][1] = cmulsub(Z[0][2], Z[1][0], Z[0][0], Z[1][2]);
    Cf[2][2] = cmulsub(Z[0][0], Z[1][1], Z[0][1], Z[1][0]);
    R dr = R(0), di = R(0), tr = R(0), ti = R(0);
#pragma unroll
    for (int j = 0; j < 3; j++) {
        dr += Z[0][j].r * Cf[0][j].r - Z[0][j].i * Cf[0][j].i;
        di += Z[0][j].r * Cf[0][j].i + Z[0][j].i * Cf[0][j].r;
    }
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            tr += Cf[m][j].r * Zd[m][j].r - Cf[m][j].i * Zd[m][j].i;
            ti += Cf[m][j].r * Zd[m][j].i + Cf[m][j].i * Zd[m][j].r;
        }
    const R idn = Real<R>::rcp_pos_(dr * dr + di * di);
    // gamma = sg grad c . P^ + (tr / det) / 2
    const R gr = sg * (g[0] * Ph[0] + g[1] * Ph[1] + g[2] * Ph[2]) + R(0.5) * (tr * dr + ti * di) * idn;
    const R gi = R(0.5) * (ti * dr - tr * di) * idn;
    const R a0r = y[F_A0], a0i = y[F_A0 + 1];
    if (WAVE == 0) {
        f[F_A0] = gr * a0r - gi * a0i;
        f[F_A0 + 1] = gr * a0i + gi * a0r;
        f[F_A1] = R(0);
        f[F_A1 + 1] = R(0);
    } else {
        R Nsv[3], Nsh[3], ivn;
        s_frame<R>(P, ref_e1, Nsv, Nsh, &ivn);
        const R *Pd = f + F_P;
        R ePd0, ePd1, ePd2;
        if (ref_e1) {
            ePd0 = R(0);
            ePd1 = -Pd[2];
            ePd2 = Pd[1];
        } else {
            ePd0 = -Pd[1];
            ePd1 = Pd[0];
            ePd2 = R(0);
        }
        const R om = (ePd0 * Nsv[0] + ePd1 * Nsv[1] + ePd2 * Nsv[2]) * ivn;
        const R a1r = y[F_A1], a1i = y[F_A1 + 1];
        f[F_A0] = gr * a0r - gi * a0i - om * a1r;
        f[F_A0 + 1] = gr * a0i + gi * a0r - om * a1i;
        f[F_A1] = gr * a1r - gi * a1i + om * a0r;
        f[F_A1 + 1] = gr * a1i + gi * a1r + om * a0i;
    }
}

// The same record from the end states and only the Q, P parts of the slopes (d0, d1: 6 values each
// at offsets F_Q..F_P+2, as in the state).
template <typename R, int WAVE>
__device__ __forceinline__ void beam_record6(bool ref_e1, const R *y0, const R *d0, const R *y1, const R *d1, R dt,
                                             R th, R w, R rec[REC]);

// Reconstruction record at fraction th of a step of size dt: Q, P by cubic Hermite from
// (y0, y0', y1, y1'), amplitudes linear in th; A = w a P^ (P) or w (a_sv N_sv + a_sh N_sh) (S).
template <typename R, int WAVE>
__device__ __forceinline__ void beam_record(bool ref_e1, const R *y0, const R *d0, const R *y1, const R *d1,
                                            R dt, R th, R w, R rec[REC]) {
    const R th2 = th * th, th3 = th2 * th;
    const R h00 = R(2) * th3 - R(3) * th2 + R(1), h10 = th3 - R(2) * th2 + th;
    const R h01 = R(3) * th2 - R(2) * th3, h11 = th3 - th2;
    R P[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        rec[d] = h00 * y0[F_Q + d] + h10 * dt * d0[F_Q + d] + h01 * y1[F_Q + d] + h11 * dt * d1[F_Q + d];
        P[d] = h00 * y0[F_P + d] + h10 * dt * d0[F_P + d] + h01 * y1[F_P + d] + h11 * dt * d1[F_P + d];
        rec[3 + d] = P[d];
    }
    const R u = R(1) - th;
    const R a0r = w * (u * y0[F_A0] + th * y1[F_A0]), a0i = w * (u * y0[F_A0 + 1] + th * y1[F_A0 + 1]);
    if (WAVE == 0) {
        const R ip = Real<R>::rsqrt_(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            rec[6 + 2 * d] = a0r * P[d] * ip;
            rec[7 + 2 * d] = a0i * P[d] * ip;
        }
    } else {
        const R a1r = w * (u * y0[F_A1] + th * y1[F_A1]), a1i = w * (u * y0[F_A1 + 1] + th * y1[F_A1 + 1]);
        R Nsv[3], Nsh[3];
        s_frame<R>(P, ref_e1, Nsv, Nsh);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            rec[6 + 2 * d] = a0r * Nsv[d] + a1r * Nsh[d];
            rec[7 + 2 * d] = a0i * Nsv[d] + a1i * Nsh[d];
        }
    }
}

template <typename R, int WAVE>
__device__ __forceinline__ void beam_record6(bool ref_e1, const R *y0, const R *d0, const R *y1, const R *d1, R dt,
                                             R th, R w, R rec[REC]) {
    beam_record<R, WAVE>(ref_e1, y0, d0, y1, d1, dt, th, w, rec);   // reads only d[F_Q..F_P+2]
}

}  // namespace fga
