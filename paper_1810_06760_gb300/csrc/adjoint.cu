// Discrete adjoint of the forward solve (the paper gives none; it defers the adjoint to the
// tomography and waveform-inversion literature).  Reverse mode of: beam initialisation (its c(q)
// dependence), classical RK4 of the beam ODEs, the Hermite-interpolated records and the windowed
// Gaussian sums at receivers, for a seismogram cotangent ubar (ubar = u - d for the L2 misfit
// 1/2 sum |u - d|^2).  Output: the cotangents of the model's node fields (grid media), i.e. of the
// 10 trilinearly interpolated fields c, grad c, Hess c of the P and of the S grid.
//
// Schedule (one thread per beam throughout):
//   1. forward pass storing the state every C steps (checkpoints);
//   2. for each segment, last to first: recompute its C states from the checkpoint, then the reverse
//      steps, last to first.  A reverse step reads y_n, y_{n+1} and the running cotangent
//      ybar_{n+1}; adds the record cotangents of the step's samples (receivers and the step's
//      seismogram cotangents staged in shared memory), then runs RK4 backwards through its four
//      stages with the hand-written adjoint of dy/dt (one kernel per part, see reverse_step); writes
//      ybar_n.
//   3. the cotangent of the initial amplitudes gives dL/dc(q) through the initial-velocity term.
// Node-field cotangents are scattered with atomics through the interpolation weights (GradAcc).
#include <cmath>
#include <vector>

#include "fga_beam.cuh"
#include "gather.cuh"

namespace fga {
namespace {

template <typename R> __device__ __forceinline__ C2<R> cconj_mul(C2<R> a, C2<R> b) {  // conj(a) b
    return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r};
}
template <typename R> __device__ __forceinline__ C2<R> cadd(C2<R> a, C2<R> b) { return {a.r + b.r, a.i + b.i}; }
template <typename R> __device__ __forceinline__ C2<R> cscale(R s, C2<R> a) { return {s * a.r, s * a.i}; }
template <typename R> __device__ __forceinline__ R re_conj_mul(C2<R> a, C2<R> b) { return a.r * b.r + a.i * b.i; }
template <typename R> __device__ __forceinline__ C2<R> ld2(const R *p) { return {p[0], p[1]}; }
template <typename R> __device__ __forceinline__ void add2(R *p, C2<R> v) {
    p[0] += v.r;
    p[1] += v.i;
}

// Node-field cotangent accumulators.  FP64: atomics straight into the caller's [node][10] doubles.
// FP32: 16-byte vector atomics into a scratch grid of 3 float4 per node (fields 0-9, 2 pad), added
// to the caller's doubles at the end (3 reductions per node instead of 10 FP64 atomics).
template <typename R> struct GradAcc;
template <> struct GradAcc<double> {
    double *p;
    __device__ __forceinline__ void add(int64_t node, const double cb[10], double w) const {
#pragma unroll
        for (int f = 0; f < 10; f++) atomicAdd(p + node * 10 + f, cb[f] * w);
    }
};
template <> struct GradAcc<float> {
    float4 *p;
    __device__ __forceinline__ void add(int64_t node, const float cb[10], float w) const {
        float4 *q = p + 3 * node;
        atomicAdd(q, make_float4(cb[0] * w, cb[1] * w, cb[2] * w, cb[3] * w));
        atomicAdd(q + 1, make_float4(cb[4] * w, cb[5] * w, cb[6] * w, cb[7] * w));
        atomicAdd(q + 2, make_float4(cb[8] * w, cb[9] * w, 0.f, 0.f));
    }
};

// Deferred node cotangents: a stage adjoint records its sampling point and field cotangents (13
// reals per beam, SoA with stride cap) instead of scattering; adj_scatter_kernel later adds the
// records of one step that share a trilinear cell together and scatters each distinct cell once.
template <typename R> struct DeferAcc {
    R *p;
    int64_t cap, b;
    __device__ __forceinline__ void put(const R x[3], const R cb[10]) const {
#pragma unroll
        for (int d = 0; d < 3; d++) __stcs(p + (int64_t)d * cap + b, x[d]);
#pragma unroll
        for (int f = 0; f < 10; f++) __stcs(p + (int64_t)(3 + f) * cap + b, cb[f]);
    }
};
constexpr int DEFER_FIELDS = 13;
template <typename G> struct is_deferred { static constexpr bool value = false; };
template <typename R> struct is_deferred<DeferAcc<R>> { static constexpr bool value = true; };

// the trilinear cell of x: lower corner i[], fractions fr[], d fr/dx (zero where x is clamped)
template <typename R>
__device__ __forceinline__ void trilinear_cell(const ModelDev &M, const R x[3], int i[3], R fr[3], R dfr[3]) {
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const R ih = mp<R>(M.inv_h[d], M.finv_h[d]);
        R t = (x[d] - mp<R>(M.o[d], M.fo[d])) * ih;
        const R hi = R(M.n[d] - 1);
        dfr[d] = ih;
        if (t < R(0)) {
            t = R(0);
            dfr[d] = R(0);
        }
        if (t > hi) {
            t = hi;
            dfr[d] = R(0);
        }
        int id = (int)Real<R>::floor_(t);
        id = id > M.n[d] - 2 ? M.n[d] - 2 : id;
        i[d] = id;
        fr[d] = t - R(id);
    }
}

// ---------------------------------------------------------------------------------------------
// adjoint of the trilinear model sampling: Qb += sum_f cb_f d field_f / dQ; grad[node][f] += w cb_f
// (G = GradAcc: scattered here; G = DeferAcc: recorded for adj_scatter_kernel)
// ---------------------------------------------------------------------------------------------
template <typename R, int MED, class G>
__device__ __forceinline__ void model_vjp(const ModelDev &M, int wave, const R x[3], const R cb[10], R Qb[3],
                                          G grad) {
    if (MED != FGA_MEDIUM_GRID) return;  // constant media: no position or node dependence
    const float4 *__restrict__ Gm = wave ? M.gs : M.gp;
    int i[3];
    R fr[3], dfr[3];
    trilinear_cell<R>(M, x, i, fr, dfr);
    if constexpr (is_deferred<G>::value) grad.put(x, cb);
    const int64_t s1 = M.n[2], s0 = (int64_t)M.n[1] * M.n[2];
    const int64_t base = (int64_t)i[0] * s0 + (int64_t)i[1] * s1 + i[2];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int64_t node = base + a * s0 + b * s1 + c;
                const R w0 = a ? fr[0] : R(1) - fr[0], w1 = b ? fr[1] : R(1) - fr[1], w2 = c ? fr[2] : R(1) - fr[2];
                const R g0 = a ? dfr[0] : -dfr[0], g1 = b ? dfr[1] : -dfr[1], g2 = c ? dfr[2] : -dfr[2];
                const float4 *p = Gm + 3 * node;
                const float4 u0 = __ldg(p), u1 = __ldg(p + 1), u2 = __ldg(p + 2);
                const float v[10] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y};
                R dot = R(0);
#pragma unroll
                for (int f = 0; f < 10; f++) dot += cb[f] * (R)v[f];
                Qb[0] += dot * g0 * w1 * w2;
                Qb[1] += dot * w0 * g1 * w2;
                Qb[2] += dot * w0 * w1 * g2;
                if constexpr (!is_deferred<G>::value)
                    if (grad.p) grad.add(node, cb, w0 * w1 * w2);
            }
}

// ---------------------------------------------------------------------------------------------
// adjoint of dy/dt (the right-hand side of beam_rhs): yb += (d rhs / dy)^T fb, node-field
// cotangents to grad.  Complex cotangents follow zb = dL/dRe z + i dL/dIm z.
// ---------------------------------------------------------------------------------------------
template <typename R, int WAVE, int MED, class FB, class G>
__device__ __forceinline__ void rhs_vjp(const ModelDev &M, R sg, bool ref_e1, const R *__restrict__ y, FB fb,
                                        R *__restrict__ yb, G grad) {
    R cf[10];
    const R Q[3] = {y[F_Q], y[F_Q + 1], y[F_Q + 2]};
    model_eval<R, MED>(M, WAVE, Q, cf);
    const R c = cf[0];
    const R g[3] = {cf[1], cf[2], cf[3]};
    const R H[3][3] = {{cf[4], cf[5], cf[6]}, {cf[5], cf[7], cf[8]}, {cf[6], cf[8], cf[9]}};
    const R P[3] = {y[F_P], y[F_P + 1], y[F_P + 2]};
    const R p2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const R ip = Real<R>::rsqrt_(p2);
    const R pn = p2 * ip;   // |P| as in beam_rhs
    const R Ph[3] = {P[0] * ip, P[1] * ip, P[2] * ip};
    const R cip = c * ip;
    // forward intermediates: u = dzQ g, v = dzP P^, t3 = dzQ H, Z, Z'
    C2<R> u[3], v[3], Z[3][3], Zd[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        u[m] = {R(0), R(0)};
        v[m] = {R(0), R(0)};
#pragma unroll
        for (int l = 0; l < 3; l++) {
            u[m] = cadd(u[m], cscale(g[l], ld2(y + F_DQ + 2 * (3 * m + l))));
            v[m] = cadd(v[m], cscale(Ph[l], ld2(y + F_DP + 2 * (3 * m + l))));
        }
    }
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const C2<R> dq = ld2(y + F_DQ + 2 * (3 * m + j)), dp = ld2(y + F_DP + 2 * (3 * m + j));
            C2<R> t3 = {R(0), R(0)};
#pragma unroll
            for (int l = 0; l < 3; l++) t3 = cadd(t3, cscale(H[l][j], ld2(y + F_DQ + 2 * (3 * m + l))));
            const C2<R> fdq = cscale(sg, cadd(cadd(cscale(Ph[j], u[m]), cscale(cip, dp)), cscale(-cip * Ph[j], v[m])));
            const C2<R> fdp = cscale(-sg, cadd(cscale(pn, t3), cscale(g[j], v[m])));
            Z[m][j] = {dq.r - dp.i, dq.i + dp.r};
            Zd[m][j] = {fdq.r - fdp.i, fdq.i + fdp.r};
        }
    // Z^-1 = cof(Z)^T / det Z
    C2<R> Zi[3][3];
    {
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
        C2<R> det = {R(0), R(0)};
#pragma unroll
        for (int j = 0; j < 3; j++) det = cadd(det, cmul(Z[0][j], Cf[0][j]));
        const R idn = Real<R>::rcp_pos_(det.r * det.r + det.i * det.i);
        const C2<R> idet = {det.r * idn, -det.i * idn};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) Zi[a][b] = cmul(Cf[b][a], idet);
    }
    C2<R> tr = {R(0), R(0)};
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 3; j++) tr = cadd(tr, cmul(Zi[j][m], Zd[m][j]));
    const C2<R> gam = {sg * (g[0] * Ph[0] + g[1] * Ph[1] + g[2] * Ph[2]) + R(0.5) * tr.r, R(0.5) * tr.i};

    // ---- reverse sweep ----
    R cb[10];
#pragma unroll
    for (int f = 0; f < 10; f++) cb[f] = R(0);
    R Phb[3] = {R(0), R(0), R(0)}, Pb[3] = {R(0), R(0), R(0)}, pnb = R(0), cipb = R(0);
    R fPb[3] = {fb(F_P), fb(F_P + 1), fb(F_P + 2)};
    const C2<R> a0 = ld2(y + F_A0), fa0 = {fb(F_A0), fb(F_A0 + 1)};
    C2<R> gamb;
    if (WAVE == 0) {
        add2(yb + F_A0, cconj_mul(gam, fa0));
        gamb = cconj_mul(a0, fa0);
    } else {
        // omega = -s1 s2 / D, s1 = P'.(e x P), s2 = e.P, D = |P|^3 - s2^2 |P|,  P' = -sg |P| g
        const C2<R> a1 = ld2(y + F_A1), fa1 = {fb(F_A1), fb(F_A1 + 1)};
        R exP[3], e[3];
        if (ref_e1) {
            e[0] = R(1); e[1] = R(0); e[2] = R(0);
            exP[0] = R(0); exP[1] = -P[2]; exP[2] = P[1];
        } else {
            e[0] = R(0); e[1] = R(0); e[2] = R(1);
            exP[0] = -P[1]; exP[1] = P[0]; exP[2] = R(0);
        }
        const R fP[3] = {-sg * pn * g[0], -sg * pn * g[1], -sg * pn * g[2]};
        const R s1 = fP[0] * exP[0] + fP[1] * exP[1] + fP[2] * exP[2];
        const R s2 = ref_e1 ? P[0] : P[2];
        const R D = pn * pn * pn - s2 * s2 * pn;   // |P| |e x P|^2 > 0 (the S frame keeps e off P)
        const R iD = Real<R>::rcp_pos_(D);
        const R om = -s1 * s2 * iD;
        // a0' = gam a0 - om a1, a1' = gam a1 + om a0
        add2(yb + F_A0, cadd(cconj_mul(gam, fa0), cscale(om, fa1)));
        add2(yb + F_A1, cadd(cconj_mul(gam, fa1), cscale(-om, fa0)));
        gamb = cadd(cconj_mul(a0, fa0), cconj_mul(a1, fa1));
        const R omb = -re_conj_mul(a1, fa0) + re_conj_mul(a0, fa1);
        // fP x e
        R fPxe[3];
        if (ref_e1) {
            fPxe[0] = R(0); fPxe[1] = fP[2]; fPxe[2] = -fP[1];
        } else {
            fPxe[0] = fP[1]; fPxe[1] = -fP[0]; fPxe[2] = R(0);
        }
        const R k1 = -s2 * iD, k2 = -s1 * iD, k3 = s1 * s2 * iD * iD;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            fPb[d] += omb * k1 * exP[d];
            const R dD = R(3) * pn * P[d] - R(2) * s2 * pn * e[d] - s2 * s2 * P[d] * ip;
            Pb[d] += omb * (k1 * fPxe[d] + k2 * e[d] + k3 * dD);
        }
    }
    // gamma = sg g.P^ + tr/2
#pragma unroll
    for (int d = 0; d < 3; d++) {
        cb[1 + d] += sg * Ph[d] * gamb.r;
        Phb[d] += sg * g[d] * gamb.r;
    }
    const C2<R> trb = cscale(R(0.5), gamb);
    // tr = sum_mj Zi_jm Z'_mj: Z'b_mj = conj(Zi_jm) trb, Zb_mj = -conj((Zi Z' Zi)_jm) trb
    C2<R> fDQb[3][3], fDPb[3][3];
    {
        C2<R> ZdZi[3][3];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                C2<R> s = {R(0), R(0)};
#pragma unroll
                for (int q = 0; q < 3; q++) s = cadd(s, cmul(Zd[a][q], Zi[q][b]));
                ZdZi[a][b] = s;
            }
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                C2<R> M3 = {R(0), R(0)};  // (Zi Z' Zi)_jm
#pragma unroll
                for (int a = 0; a < 3; a++) M3 = cadd(M3, cmul(Zi[j][a], ZdZi[a][m]));
                const C2<R> zdb = cconj_mul(Zi[j][m], trb);
                const C2<R> zb = cscale(R(-1), cconj_mul(M3, trb));
                const int e = 2 * (3 * m + j);
                // Z = dzQ + i dzP: dzQ_b += zb, dzP_b += -i zb; likewise for Z'
                fDQb[m][j] = cadd(C2<R>{fb(F_DQ + e), fb(F_DQ + e + 1)}, zdb);
                fDPb[m][j] = cadd(C2<R>{fb(F_DP + e), fb(F_DP + e + 1)}, C2<R>{zdb.i, -zdb.r});
                add2(yb + F_DQ + e, zb);
                add2(yb + F_DP + e, {zb.i, -zb.r});
            }
    }
    // dzP' = -sg (|P| dzQ H + v g^T)
    C2<R> ub[3] = {{R(0), R(0)}, {R(0), R(0)}, {R(0), R(0)}}, vb[3] = {{R(0), R(0)}, {R(0), R(0)}, {R(0), R(0)}};
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const C2<R> b = fDPb[m][j];
            C2<R> t3 = {R(0), R(0)};
#pragma unroll
            for (int l = 0; l < 3; l++) t3 = cadd(t3, cscale(H[l][j], ld2(y + F_DQ + 2 * (3 * m + l))));
            pnb += -sg * re_conj_mul(t3, b);
            vb[m] = cadd(vb[m], cscale(-sg * g[j], b));
            cb[1 + j] += -sg * re_conj_mul(v[m], b);
            const C2<R> t3b = cscale(-sg * pn, b);
#pragma unroll
            for (int l = 0; l < 3; l++) {
                add2(yb + F_DQ + 2 * (3 * m + l), cscale(H[l][j], t3b));
                const R hb = re_conj_mul(ld2(y + F_DQ + 2 * (3 * m + l)), t3b);
                // H_lj is field 4 + (symmetric index)
                const int hi = (l == 0) ? 4 + j : (l == 1 ? (j == 0 ? 5 : 6 + j) : (j == 0 ? 6 : (j == 1 ? 8 : 9)));
                cb[hi] += hb;
            }
        }
    // dzQ' = sg (u P^T + (c/|P|) dzP - (c/|P|) v P^T)
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const C2<R> b = fDQb[m][j];
            const C2<R> dp = ld2(y + F_DP + 2 * (3 * m + j));
            ub[m] = cadd(ub[m], cscale(sg * Ph[j], b));
            add2(yb + F_DP + 2 * (3 * m + j), cscale(sg * cip, b));
            vb[m] = cadd(vb[m], cscale(-sg * cip * Ph[j], b));
            cipb += sg * re_conj_mul({dp.r - v[m].r * Ph[j], dp.i - v[m].i * Ph[j]}, b);
            Phb[j] += sg * re_conj_mul({u[m].r - cip * v[m].r, u[m].i - cip * v[m].i}, b);
        }
    // u = dzQ g, v = dzP P^
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
        for (int l = 0; l < 3; l++) {
            add2(yb + F_DQ + 2 * (3 * m + l), cscale(g[l], ub[m]));
            cb[1 + l] += re_conj_mul(ld2(y + F_DQ + 2 * (3 * m + l)), ub[m]);
            add2(yb + F_DP + 2 * (3 * m + l), cscale(Ph[l], vb[m]));
            Phb[l] += re_conj_mul(ld2(y + F_DP + 2 * (3 * m + l)), vb[m]);
        }
    // P' = -sg |P| g, Q' = sg c P^
#pragma unroll
    for (int d = 0; d < 3; d++) {
        pnb += -sg * g[d] * fPb[d];
        cb[1 + d] += -sg * pn * fPb[d];
        const R fq = fb(F_Q + d);
        cb[0] += sg * Ph[d] * fq;
        Phb[d] += sg * c * fq;
    }
    cb[0] += ip * cipb;
    pnb += -c * ip * ip * cipb;
    const R phd = Phb[0] * Ph[0] + Phb[1] * Ph[1] + Phb[2] * Ph[2];
#pragma unroll
    for (int d = 0; d < 3; d++) yb[F_P + d] += Pb[d] + (Phb[d] - Ph[d] * phd) * ip + pnb * Ph[d];
    R Qb[3] = {R(0), R(0), R(0)};
    model_vjp<R, MED>(M, WAVE, Q, cb, Qb, grad);
#pragma unroll
    for (int d = 0; d < 3; d++) yb[F_Q + d] += Qb[d];
}

// adjoint of the S frame: Pb += cotangent of P from those of N_sv and N_sh
template <typename R>
__device__ __forceinline__ void s_frame_vjp(const R P[3], bool ref_e1, const R Nsvb[3], const R Nshb[3], R Pb[3]) {
    R Nsv[3], Nsh[3], iv;
    s_frame<R>(P, ref_e1, Nsv, Nsh, &iv);
    const R ip = Real<R>::rsqrt_(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    const R Ph[3] = {P[0] * ip, P[1] * ip, P[2] * ip};
    // N_sv = N_sh x P^: N_sh_b += P^ x N_sv_b, P^_b = N_sv_b x N_sh
    const R nb[3] = {Nshb[0] + Ph[1] * Nsvb[2] - Ph[2] * Nsvb[1], Nshb[1] + Ph[2] * Nsvb[0] - Ph[0] * Nsvb[2],
                     Nshb[2] + Ph[0] * Nsvb[1] - Ph[1] * Nsvb[0]};
    const R phb[3] = {Nsvb[1] * Nsh[2] - Nsvb[2] * Nsh[1], Nsvb[2] * Nsh[0] - Nsvb[0] * Nsh[2],
                      Nsvb[0] * Nsh[1] - Nsvb[1] * Nsh[0]};
    const R s1 = Nsh[0] * nb[0] + Nsh[1] * nb[1] + Nsh[2] * nb[2];
    const R vb[3] = {(nb[0] - Nsh[0] * s1) * iv, (nb[1] - Nsh[1] * s1) * iv, (nb[2] - Nsh[2] * s1) * iv};
    // v = e x P: P_b += v_b x e
    if (ref_e1) {
        Pb[1] += vb[2];
        Pb[2] -= vb[1];
    } else {
        Pb[0] += vb[1];
        Pb[1] -= vb[0];
    }
    const R s2 = Ph[0] * phb[0] + Ph[1] * phb[1] + Ph[2] * phb[2];
#pragma unroll
    for (int d = 0; d < 3; d++) Pb[d] += (phb[d] - Ph[d] * s2) * ip;
}

// cotangent of a record from the cotangents of one sample's receivers (shared memory):
// u(x) += A exp(phi), phi = i k P.(x - Q) - k |x - Q|^2 / 2 inside the window
template <typename R>
__device__ __forceinline__ void gauss_vjp(const R rec[REC], const R *__restrict__ xs, const R *__restrict__ us, int nrx,
                                          R k, R rw2, R rb[REC]) {
    R Ab[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    R Sr = R(0), Si = R(0), Vr[3] = {R(0), R(0), R(0)}, Vi[3] = {R(0), R(0), R(0)};
    const R hk = R(-0.5) * k;
    for (int i = 0; i < nrx; i++) {
        const R d0 = xs[3 * i] - rec[0], d1 = xs[3 * i + 1] - rec[1], d2 = xs[3 * i + 2] - rec[2];
        const R r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 > rw2) continue;
        R er, ei;
        gauss_phase_exp<R>(k * (rec[3] * d0 + rec[4] * d1 + rec[5] * d2), hk * r2, &er, &ei);
        const R *u = us + 6 * i;
        // Ab += conj(E) u;  Eb = sum conj(A) u;  phib = conj(E) Eb
        R ebr = R(0), ebi = R(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const R ur = u[2 * d], ui = u[2 * d + 1];
            Ab[2 * d] = fma(er, ur, fma(ei, ui, Ab[2 * d]));
            Ab[2 * d + 1] = fma(er, ui, fma(-ei, ur, Ab[2 * d + 1]));
            const R ar = rec[6 + 2 * d], ai = rec[7 + 2 * d];
            ebr = fma(ar, ur, fma(ai, ui, ebr));
            ebi = fma(ar, ui, fma(-ai, ur, ebi));
        }
        const R pr = er * ebr + ei * ebi, pi = er * ebi - ei * ebr;
        Sr += pr;
        Si += pi;
        Vr[0] = fma(d0, pr, Vr[0]);
        Vr[1] = fma(d1, pr, Vr[1]);
        Vr[2] = fma(d2, pr, Vr[2]);
        Vi[0] = fma(d0, pi, Vi[0]);
        Vi[1] = fma(d1, pi, Vi[1]);
        Vi[2] = fma(d2, pi, Vi[2]);
    }
    // d phi/dP = i k dx, d phi/dQ = -i k P + k dx
#pragma unroll
    for (int d = 0; d < 3; d++) {
        rb[d] = k * (Vr[d] - rec[3 + d] * Si);
        rb[3 + d] = k * Vi[d];
        rb[6 + 2 * d] = Ab[2 * d];
        rb[7 + 2 * d] = Ab[2 * d + 1];
    }
}

// adjoint of beam_record: record cotangent -> cotangents of y0, y1 (full) and of y0', y1' (Q, P)
template <typename R, int WAVE>
__device__ __forceinline__ void record_vjp(bool ref_e1, const R *y0, const R *d0, const R *y1, const R *d1, R dt,
                                           R th, R w, const R rb[REC], R *y0b, R f0b[6], R *y1b, R f1b[6]) {
    const R th2 = th * th, th3 = th2 * th;
    const R h00 = R(2) * th3 - R(3) * th2 + R(1), h10 = th3 - R(2) * th2 + th;
    const R h01 = R(3) * th2 - R(2) * th3, h11 = th3 - th2;
    R P[3], Pb[3] = {rb[3], rb[4], rb[5]};
#pragma unroll
    for (int d = 0; d < 3; d++)
        P[d] = h00 * y0[F_P + d] + h10 * dt * d0[F_P + d] + h01 * y1[F_P + d] + h11 * dt * d1[F_P + d];
    const R uu = R(1) - th;
    const C2<R> a0 = {uu * y0[F_A0] + th * y1[F_A0], uu * y0[F_A0 + 1] + th * y1[F_A0 + 1]};
    C2<R> ab0 = {R(0), R(0)}, ab1 = {R(0), R(0)};
    if (WAVE == 0) {
        const R ip = Real<R>::rsqrt_(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
        const R Ph[3] = {P[0] * ip, P[1] * ip, P[2] * ip};
        R Phb[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const C2<R> A = {rb[6 + 2 * d], rb[7 + 2 * d]};
            ab0 = cadd(ab0, cscale(w * Ph[d], A));
            Phb[d] = w * re_conj_mul(a0, A);
        }
        const R s = Ph[0] * Phb[0] + Ph[1] * Phb[1] + Ph[2] * Phb[2];
#pragma unroll
        for (int d = 0; d < 3; d++) Pb[d] += (Phb[d] - Ph[d] * s) * ip;
    } else {
        const C2<R> a1 = {uu * y0[F_A1] + th * y1[F_A1], uu * y0[F_A1 + 1] + th * y1[F_A1 + 1]};
        R Nsv[3], Nsh[3], Nsvb[3], Nshb[3];
        s_frame<R>(P, ref_e1, Nsv, Nsh);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const C2<R> A = {rb[6 + 2 * d], rb[7 + 2 * d]};
            ab0 = cadd(ab0, cscale(w * Nsv[d], A));
            ab1 = cadd(ab1, cscale(w * Nsh[d], A));
            Nsvb[d] = w * re_conj_mul(a0, A);
            Nshb[d] = w * re_conj_mul(a1, A);
        }
        s_frame_vjp<R>(P, ref_e1, Nsvb, Nshb, Pb);
        add2(y0b + F_A1, cscale(uu, ab1));
        add2(y1b + F_A1, cscale(th, ab1));
    }
    add2(y0b + F_A0, cscale(uu, ab0));
    add2(y1b + F_A0, cscale(th, ab0));
#pragma unroll
    for (int d = 0; d < 3; d++) {
        y0b[F_Q + d] += h00 * rb[d];
        f0b[d] += h10 * dt * rb[d];
        y1b[F_Q + d] += h01 * rb[d];
        f1b[d] += h11 * dt * rb[d];
        y0b[F_P + d] += h00 * Pb[d];
        f0b[3 + d] += h10 * dt * Pb[d];
        y1b[F_P + d] += h01 * Pb[d];
        f1b[3 + d] += h11 * dt * Pb[d];
    }
}

// Beam states, slopes and cotangents stream through once per launch (hundreds of MB): evict-first
// loads and stores keep the model grids and the node-cotangent scratch resident in L2.
template <typename R> __device__ __forceinline__ void load_state(const R *__restrict__ S, int64_t cap, int64_t b, R *y) {
#pragma unroll
    for (int f = 0; f < NF; f++) y[f] = __ldcs(S + (int64_t)f * cap + b);
}
template <typename R> __device__ __forceinline__ void store_state(R *__restrict__ S, int64_t cap, int64_t b, const R *y) {
#pragma unroll
    for (int f = 0; f < NF; f++) __stcs(S + (int64_t)f * cap + b, y[f]);
}

// Forward RK4 from src (SoA, stride cap) for nsteps; the state after step s (1-based) is stored in
// slot s/every of dst when s is a multiple of every (slot stride slot).
template <typename R, int WAVE, int MED>
__global__ void __launch_bounds__(128) adj_forward_kernel(ModelDev M, const R *__restrict__ src, R *__restrict__ dst,
                                                         int64_t cap, int64_t slot, const int32_t *__restrict__ flags,
                                                         int64_t off, int64_t n, R sg, R dt, int nsteps, int every) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off + i;
    const bool e1 = (flags[b] & FL_REF_E1) != 0;
    R y[NF], k[NF], t[NF], acc[NF];
    load_state(src, cap, b, y);
    const R h = R(0.5) * dt, s6 = dt / R(6);
    for (int s = 1; s <= nsteps; s++) {
        beam_rhs<R, WAVE, MED>(M, sg, e1, y, k);
#pragma unroll
        for (int f = 0; f < NF; f++) {
            acc[f] = k[f];
            t[f] = y[f] + h * k[f];
        }
        beam_rhs<R, WAVE, MED>(M, sg, e1, t, k);
#pragma unroll
        for (int f = 0; f < NF; f++) {
            acc[f] += R(2) * k[f];
            t[f] = y[f] + h * k[f];
        }
        beam_rhs<R, WAVE, MED>(M, sg, e1, t, k);
#pragma unroll
        for (int f = 0; f < NF; f++) {
            acc[f] += R(2) * k[f];
            t[f] = y[f] + dt * k[f];
        }
        beam_rhs<R, WAVE, MED>(M, sg, e1, t, k);
#pragma unroll
        for (int f = 0; f < NF; f++) y[f] += s6 * (acc[f] + k[f]);
        if (s % every == 0) store_state(dst + (int64_t)(s / every) * slot, cap, b, y);
    }
}

// Reverse step n, split into one kernel per part so that each keeps about three 46-real arrays
// live (a single kernel holding the step's state, slopes and cotangents spilled to local memory):
//   adj_records_kernel  (steps with samples) record cotangents: ybar_{n+1} += those of y_{n+1} (with
//                       the adjoint of its slope when a sample lies inside the step); the cotangents of
//                       y_n and of k1 (Q, P) go to RB;
//   adj_stage4_kernel   recomputes the stage inputs t2 = y + h k1 and t3 = y + h k2 (stored) and
//                       t4 = y + dt k3; sb4 = (df/dy(t4))^T (dt/6 ybar_{n+1});
//   adj_stage_kernel    sb3 at t3 from dt/3 ybar_{n+1} + dt sb4, then sb2 at t2 from dt/3 ybar_{n+1} + h sb3;
//   adj_stage1_kernel   ybar_n = ybar_{n+1} + sb4 + sb3 + sb2 + RB + (df/dy(y))^T (dt/6 ybar_{n+1} + h sb2
//                       + RB's k1 part).
// All buffers are SoA with stride cap, indexed by the beam's slot.
struct StepSamples {
    int nsj, need_d1;
    float th[4];
    double thd[4];
    double lo[3], hi[3];  // bounding box of the receivers
};
constexpr int ADJ_THREADS = 128;

// RB layout: fields 0-5 = cotangent of y_n's Q, P; 6-9 = of its amplitudes; 10-15 = of k1's Q, P
constexpr int RB_FIELDS = 16;

// Cotangent of a stage slope, a ybar_{n+1} + c sb (+ the records' k1 cotangent on Q, P), formed once
// at kernel start into the thread's own column of shared memory (column stride ADJ_THREADS): all of
// its global loads go out together instead of one round trip per use inside the adjoint.
template <typename R> struct StagedBar {
    const R *p;  // &column[threadIdx.x]
    __device__ __forceinline__ R operator()(int f) const { return p[f * ADJ_THREADS]; }
};
template <typename R>
__device__ __forceinline__ StagedBar<R> stage_slope_bar(R *col, const R *yb, const R *sb, const R *rb, int64_t cap,
                                                        int64_t b, R a, R c) {
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const int64_t o = (int64_t)f * cap + b;
        R v = a * __ldcs(yb + o);
        if (sb) v += c * __ldcs(sb + o);
        if (f < 6 && rb) v += __ldcs(rb + (int64_t)(10 + f) * cap + b);
        col[f * ADJ_THREADS] = v;
    }
    return StagedBar<R>{col};
}
// cotangent held in registers on Q, P only (the records' slope term at y_{n+1})
template <typename R> struct QPBar {
    const R *v;
    __device__ __forceinline__ R operator()(int f) const { return f < 6 ? v[f] : R(0); }
};

// D1: some sample lies strictly inside the step, so the records depend on y_{n+1}'s slope as well
template <typename R, int WAVE, int MED, bool D1>
__global__ void __launch_bounds__(ADJ_THREADS) adj_records_kernel(ModelDev M, const R *__restrict__ Sn,
                                                         const R *__restrict__ Sn1, R *__restrict__ YB,
                                                         R *__restrict__ RB, int64_t cap,
                                                         const int32_t *__restrict__ flags, int64_t off, int64_t n,
                                                         R sg, R dt, R w, R k, R rw2, int nrx,
                                                         const R *__restrict__ rx, const R *__restrict__ ub,
                                                         StepSamples ss, GradAcc<R> grad) {
    extern __shared__ unsigned char smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);
    R *us = xs + 3 * nrx;
    for (int i = threadIdx.x; i < 3 * nrx; i += blockDim.x) xs[i] = rx[i];
    for (int i = threadIdx.x; i < 6 * nrx * ss.nsj; i += blockDim.x) us[i] = ub[i];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off + i;
    const bool e1 = (flags[b] & FL_REF_E1) != 0;
    R y[NF], k1[NF], y1[NF], d1[NF], y0b[NF], y1b[NF];
    load_state(Sn, cap, b, y);
    beam_rhs<R, WAVE, MED>(M, sg, e1, y, k1);
    load_state(Sn1, cap, b, y1);
    if constexpr (D1)
        beam_rhs<R, WAVE, MED>(M, sg, e1, y1, d1);
    else
#pragma unroll
        for (int f = 0; f < NF; f++) d1[f] = R(0);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        y0b[f] = R(0);
        y1b[f] = R(0);
    }
    R f0b[6] = {R(0), R(0), R(0), R(0), R(0), R(0)}, f1b[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int s = 0; s < ss.nsj; s++) {
        const R th = sizeof(R) == 8 ? (R)ss.thd[s] : (R)ss.th[s];
        R rec[REC], rb[REC];
        beam_record<R, WAVE>(e1, y, k1, y1, d1, dt, th, w, rec);
        // no receiver within the window (with a margin over rounding): the record's cotangent is zero
        R bd2 = R(0);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const R lo = (R)ss.lo[d] - rec[d], hi = rec[d] - (R)ss.hi[d];
            const R o = lo > hi ? lo : hi;
            if (o > R(0)) bd2 += o * o;
        }
        if (bd2 > rw2 * R(1.001)) continue;
        gauss_vjp<R>(rec, xs, us + (size_t)6 * nrx * s, nrx, k, rw2, rb);
        record_vjp<R, WAVE>(e1, y, k1, y1, d1, dt, th, w, rb, y0b, f0b, y1b, f1b);
    }
    if constexpr (D1) {
        rhs_vjp<R, WAVE, MED>(M, sg, e1, y1, QPBar<R>{f1b}, y1b, grad);
#pragma unroll
        for (int f = 0; f < NF; f++) YB[(int64_t)f * cap + b] += y1b[f];
    } else {
#pragma unroll
        for (int f = 0; f < 6; f++) YB[(int64_t)f * cap + b] += y1b[f];
#pragma unroll
        for (int f = 0; f < 4; f++) YB[(int64_t)(F_A0 + f) * cap + b] += y1b[F_A0 + f];
    }
#pragma unroll
    for (int f = 0; f < 6; f++) {
        RB[(int64_t)f * cap + b] = y0b[f];
        RB[(int64_t)(10 + f) * cap + b] = f0b[f];
    }
#pragma unroll
    for (int f = 0; f < 4; f++) RB[(int64_t)(6 + f) * cap + b] = y0b[F_A0 + f];
}

template <typename R, int WAVE, int MED>
__global__ void __launch_bounds__(ADJ_THREADS) adj_stage4_kernel(ModelDev M, const R *__restrict__ Sn,
                                                        const R *__restrict__ YB, R *__restrict__ T2,
                                                        R *__restrict__ T3, R *__restrict__ SB4, int64_t cap,
                                                        const int32_t *__restrict__ flags, int64_t off, int64_t n,
                                                        R sg, R dt, R *__restrict__ CBr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off + i;
    const bool e1 = (flags[b] & FL_REF_E1) != 0;
    const DeferAcc<R> grad{CBr, cap, b};
    __shared__ R col[NF * ADJ_THREADS];
    const StagedBar<R> fb = stage_slope_bar<R>(col + threadIdx.x, YB, nullptr, nullptr, cap, b, dt / R(6), R(0));
    R y[NF], kk[NF], t[NF];
    load_state(Sn, cap, b, y);
    const R h = R(0.5) * dt;
    beam_rhs<R, WAVE, MED>(M, sg, e1, y, kk);
#pragma unroll
    for (int f = 0; f < NF; f++) t[f] = y[f] + h * kk[f];
    store_state(T2, cap, b, t);
    beam_rhs<R, WAVE, MED>(M, sg, e1, t, kk);
#pragma unroll
    for (int f = 0; f < NF; f++) t[f] = y[f] + h * kk[f];
    store_state(T3, cap, b, t);
    beam_rhs<R, WAVE, MED>(M, sg, e1, t, kk);
#pragma unroll
    for (int f = 0; f < NF; f++) t[f] = y[f] + dt * kk[f];
    R sb[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) sb[f] = R(0);
    rhs_vjp<R, WAVE, MED>(M, sg, e1, t, fb, sb, grad);
    store_state(SB4, cap, b, sb);
}

// sb_out = (df/dy(t))^T (a ybar_{n+1} + c sb_in)
template <typename R, int WAVE, int MED>
__global__ void __launch_bounds__(ADJ_THREADS) adj_stage_kernel(ModelDev M, const R *__restrict__ T, const R *__restrict__ YB,
                                                       const R *__restrict__ SBin, R *__restrict__ SBout, int64_t cap,
                                                       const int32_t *__restrict__ flags, int64_t off, int64_t n,
                                                       R sg, R a, R c, R *__restrict__ CBr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off + i;
    const bool e1 = (flags[b] & FL_REF_E1) != 0;
    const DeferAcc<R> grad{CBr, cap, b};
    __shared__ R col[NF * ADJ_THREADS];
    const StagedBar<R> fb = stage_slope_bar<R>(col + threadIdx.x, YB, SBin, nullptr, cap, b, a, c);
    R t[NF], sb[NF];
    load_state(T, cap, b, t);
#pragma unroll
    for (int f = 0; f < NF; f++) sb[f] = R(0);
    rhs_vjp<R, WAVE, MED>(M, sg, e1, t, fb, sb, grad);
    store_state(SBout, cap, b, sb);
}

// YB: ybar_{n+1} on entry, ybar_n on exit (read and written by the same thread only)
template <typename R, int WAVE, int MED>
__global__ void __launch_bounds__(ADJ_THREADS) adj_stage1_kernel(ModelDev M, const R *__restrict__ Sn, R *YB,
                                                        const R *__restrict__ SB4, const R *__restrict__ SB3,
                                                        const R *__restrict__ SB2, const R *__restrict__ RB,
                                                        int64_t cap, const int32_t *__restrict__ flags, int64_t off,
                                                        int64_t n, R sg, R dt, R *__restrict__ CBr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off + i;
    const bool e1 = (flags[b] & FL_REF_E1) != 0;
    const DeferAcc<R> grad{CBr, cap, b};
    __shared__ R col[NF * ADJ_THREADS];
    const StagedBar<R> fb = stage_slope_bar<R>(col + threadIdx.x, YB, SB2, RB, cap, b, dt / R(6), R(0.5) * dt);
    R y[NF], yb[NF];
    load_state(Sn, cap, b, y);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        const int64_t o = (int64_t)f * cap + b;
        yb[f] = __ldcs(YB + o) + __ldcs(SB4 + o) + __ldcs(SB3 + o) + __ldcs(SB2 + o);
    }
    if (RB) {
#pragma unroll
        for (int f = 0; f < 6; f++) yb[f] += RB[(int64_t)f * cap + b];
#pragma unroll
        for (int f = 0; f < 4; f++) yb[F_A0 + f] += RB[(int64_t)(6 + f) * cap + b];
    }
    rhs_vjp<R, WAVE, MED>(M, sg, e1, y, fb, yb, grad);
    store_state(YB, cap, b, yb);
}

// Node cotangents of the last few reverse steps: nrec stage records (DEFER_FIELDS reals each, record r
// at CB + r * DEFER_FIELDS * cap), ordered along the beam's path (consecutive stage inputs lie within
// dt c / 2 of each other, a fraction of a cell).  The records are summed, with their trilinear weights,
// into the 8 x 10 cotangents of one open cell; the cell is scattered only when the path leaves it, so
// a beam touches each cell of its path about once per call instead of once per stage.
template <typename R, int WAVE>
__global__ void __launch_bounds__(ADJ_THREADS) adj_scatter_kernel(ModelDev M, const R *__restrict__ CB, int nrec,
                                                                  int64_t cap, int64_t off, int64_t n,
                                                                  GradAcc<R> grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !grad.p) return;
    const int64_t b = off + i;
    const int64_t s1 = M.n[2], s0 = (int64_t)M.n[1] * M.n[2];
    R acc[8][10];
    int64_t open = -1;
    auto flush = [&]() {
#pragma unroll
        for (int c = 0; c < 8; c++) grad.add(open + (c >> 2) * s0 + ((c >> 1) & 1) * s1 + (c & 1), acc[c], R(1));
    };
    for (int r = 0; r < nrec; r++) {
        const R *rp = CB + (int64_t)r * DEFER_FIELDS * cap + b;
        const R x[3] = {__ldcs(rp), __ldcs(rp + cap), __ldcs(rp + 2 * cap)};
        R cb[10];
#pragma unroll
        for (int f = 0; f < 10; f++) cb[f] = __ldcs(rp + (int64_t)(3 + f) * cap);
        int id[3];
        R fr[3], dfr[3];
        trilinear_cell<R>(M, x, id, fr, dfr);
        const int64_t base = (int64_t)id[0] * s0 + (int64_t)id[1] * s1 + id[2];
        if (base != open) {
            if (open >= 0) flush();
            open = base;
#pragma unroll
            for (int c = 0; c < 8; c++)
#pragma unroll
                for (int f = 0; f < 10; f++) acc[c][f] = R(0);
        }
#pragma unroll
        for (int c = 0; c < 8; c++) {
            const R w = ((c >> 2) ? fr[0] : R(1) - fr[0]) * (((c >> 1) & 1) ? fr[1] : R(1) - fr[1]) *
                        ((c & 1) ? fr[2] : R(1) - fr[2]);
#pragma unroll
            for (int f = 0; f < 10; f++) acc[c][f] += cb[f] * w;
        }
    }
    if (open >= 0) flush();
}

// dL/dc(q) of the initial amplitudes: a = 2^{3/2}(F.n +- i G.n/(k c(q) |p|))/2, so da/dc = -a_G/c with
// a_G the amplitude made from G alone (amplitudes of beams decomposed from (0, g))
template <typename R, int WAVE, int MED>
__global__ void __launch_bounds__(128) adj_init_kernel(ModelDev M, const R *__restrict__ S0, const R *__restrict__ SG,
                                                      const R *__restrict__ YB, int64_t cap, int64_t off, int64_t n,
                                                      GradAcc<R> grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = off + i;
    const R q[3] = {S0[(int64_t)F_Q * cap + b], S0[(int64_t)(F_Q + 1) * cap + b], S0[(int64_t)(F_Q + 2) * cap + b]};
    R cf[10];
    model_eval<R, MED>(M, WAVE, q, cf);
    R s = SG[(int64_t)F_A0 * cap + b] * YB[(int64_t)F_A0 * cap + b] +
          SG[(int64_t)(F_A0 + 1) * cap + b] * YB[(int64_t)(F_A0 + 1) * cap + b];
    if (WAVE)
        s += SG[(int64_t)F_A1 * cap + b] * YB[(int64_t)F_A1 * cap + b] +
             SG[(int64_t)(F_A1 + 1) * cap + b] * YB[(int64_t)(F_A1 + 1) * cap + b];
    R cb[10];
#pragma unroll
    for (int f = 0; f < 10; f++) cb[f] = R(0);
    cb[0] = -s / cf[0];
    R qb[3] = {R(0), R(0), R(0)};
    model_vjp<R, MED>(M, WAVE, q, cb, qb, grad);
}

// FP32 scratch grid (3 float4 per node) -> caller's FP64 [node][10]
__global__ void add_scratch_kernel(const float4 *__restrict__ src, double *__restrict__ dst, int64_t nn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const float4 a = src[3 * i], b = src[3 * i + 1], c = src[3 * i + 2];
    double *d = dst + i * 10;
    d[0] += a.x;
    d[1] += a.y;
    d[2] += a.z;
    d[3] += a.w;
    d[4] += b.x;
    d[5] += b.y;
    d[6] += b.z;
    d[7] += b.w;
    d[8] += c.x;
    d[9] += c.y;
}

template <typename R> struct AccSetup;
template <> struct AccSetup<double> {
    static fga_status make(double *g, int64_t, ScopedDevBuf &, cudaStream_t, GradAcc<double> &a) {
        a.p = g;
        return FGA_OK;
    }
    static fga_status finish(const ScopedDevBuf &, double *, int64_t, cudaStream_t) { return FGA_OK; }
};
template <> struct AccSetup<float> {
    static fga_status make(double *g, int64_t nn, ScopedDevBuf &buf, cudaStream_t s, GradAcc<float> &a) {
        a.p = nullptr;
        if (!g || nn == 0) return FGA_OK;
        FGA_TRY(buf.ensure(sizeof(float4) * 3 * (size_t)nn));
        FGA_CUDA(cudaMemsetAsync(buf.p, 0, sizeof(float4) * 3 * (size_t)nn, s));
        a.p = buf.as<float4>();
        return FGA_OK;
    }
    static fga_status finish(const ScopedDevBuf &buf, double *g, int64_t nn, cudaStream_t s) {
        if (!g || nn == 0 || !buf.p) return FGA_OK;
        add_scratch_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(buf.as<float4>(), g, nn);
        FGA_CUDA(cudaGetLastError());
        return FGA_OK;
    }
};

// Reverse steps whose node cotangents are scattered together (the records of SCATTER_STEPS steps).
constexpr int SCATTER_STEPS = 8;

// One reverse step of one class (beams off .. off+n-1).  RS: 4 state slots, RB_FIELDS fields, then
// 4 SCATTER_STEPS deferred-cotangent records.  The step is the jst-th (0-based) since the last scatter;
// scatter: scatter the records of steps 0..jst after it.
template <typename R, int WAVE, int MED>
fga_status reverse_step(const ModelDev &dev, const R *Sn, const R *Sn1, R *YB, R *RS, int64_t cap, int64_t slot,
                        const int32_t *fl, int64_t off, int64_t nc, R sg, R dt, R w, R k, R rw2, int nrx,
                        const R *rx, const R *ubs, const StepSamples &ss, size_t smem, GradAcc<R> gr, int jst,
                        bool scatter, cudaStream_t s) {
    R *T2 = RS, *T3 = RS + slot, *SB4 = RS + 2 * slot, *SB3 = RS + 3 * slot, *RB = RS + 4 * slot;
    R *SB2 = T3;  // t3 is dead once sb3 is formed
    const int64_t rst = (int64_t)DEFER_FIELDS * cap;
    // records in path order (latest first): step j holds stage 4, 3, 2, 1 at records 4j .. 4j+3
    R *CB0 = RB + (int64_t)RB_FIELDS * cap, *CB = CB0 + (int64_t)(4 * jst) * rst;
    const unsigned blocks = (unsigned)((nc + ADJ_THREADS - 1) / ADJ_THREADS);
    ProfScope ps(P_ADJ_REV, s);
    if (ss.nsj > 0) {
        auto kern = ss.need_d1 ? adj_records_kernel<R, WAVE, MED, true> : adj_records_kernel<R, WAVE, MED, false>;
        if (smem > 48 * 1024)
            FGA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<blocks, ADJ_THREADS, smem, s>>>(dev, Sn, Sn1, YB, RB, cap, fl, off, nc, sg, dt, w, k, rw2, nrx, rx, ubs, ss, gr);
    }
    adj_stage4_kernel<R, WAVE, MED><<<blocks, ADJ_THREADS, 0, s>>>(dev, Sn, YB, T2, T3, SB4, cap, fl, off, nc, sg, dt,
                                                                  CB);
    adj_stage_kernel<R, WAVE, MED><<<blocks, ADJ_THREADS, 0, s>>>(dev, T3, YB, SB4, SB3, cap, fl, off, nc, sg, dt / R(3), dt,
                                                                 CB + rst);
    adj_stage_kernel<R, WAVE, MED><<<blocks, ADJ_THREADS, 0, s>>>(dev, T2, YB, SB3, SB2, cap, fl, off, nc, sg, dt / R(3),
                                                                 R(0.5) * dt, CB + 2 * rst);
    adj_stage1_kernel<R, WAVE, MED><<<blocks, ADJ_THREADS, 0, s>>>(dev, Sn, YB, SB4, SB3, SB2, ss.nsj > 0 ? RB : nullptr,
                                                                  cap, fl, off, nc, sg, dt, CB + 3 * rst);
    if (MED == FGA_MEDIUM_GRID && scatter)
        adj_scatter_kernel<R, WAVE><<<blocks, ADJ_THREADS, 0, s>>>(dev, CB0, 4 * (jst + 1), cap, off, nc, gr);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

template <typename R, int MED>
fga_status run_vjp(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd, fga_beams *b,
                   fga_beams *bg, const std::vector<int> &sstep, const std::vector<double> &sth, const void *ubar,
                   double *grad_p, double *grad_s, int C, cudaStream_t s) {
    const int64_t cap = b->cap, slot = (int64_t)NF * cap;
    const int N = sd->nsteps;
    const int nseg = (N + C - 1) / C;
    const int64_t nrx = sd->n_rx;
    const double rw = sd->rw > 0 ? sd->rw : 6.0 / std::sqrt(b->k);
    ScopedDevBuf ck, seg, yb, rxd;
    FGA_TRY(ck.ensure(sizeof(R) * (size_t)slot * (size_t)(nseg + 1)));
    FGA_TRY(seg.ensure(sizeof(R) * (size_t)slot * (size_t)(C + 1)));
    FGA_TRY(yb.ensure(sizeof(R) * (size_t)slot));
    FGA_TRY(rxd.ensure(sizeof(R) * 3 * (size_t)std::max<int64_t>(nrx, 1)));
    double box_lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, box_hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
    {
        std::vector<double> rh((size_t)(3 * nrx));
        if (nrx > 0) FGA_CUDA(cudaMemcpyAsync(rh.data(), sd->rx, 8 * rh.size(), cudaMemcpyDeviceToHost, s));
        FGA_CUDA(cudaStreamSynchronize(s));
        std::vector<R> rr(rh.begin(), rh.end());
        for (int64_t r = 0; r < nrx; r++)
            for (int d = 0; d < 3; d++) {
                box_lo[d] = std::min(box_lo[d], (double)rr[(size_t)(3 * r + d)]);
                box_hi[d] = std::max(box_hi[d], (double)rr[(size_t)(3 * r + d)]);
            }
        if (nrx > 0) FGA_CUDA(cudaMemcpyAsync(rxd.p, rr.data(), sizeof(R) * rr.size(), cudaMemcpyHostToDevice, s));
        FGA_CUDA(cudaStreamSynchronize(s));
    }
    // reverse-step scratch: t2, t3 (t3's slot then holds sb2), sb4, sb3, RB_FIELDS record fields and the
    // deferred node cotangents of SCATTER_STEPS steps
    ScopedDevBuf rs;
    FGA_TRY(rs.ensure(sizeof(R) *
                      ((size_t)slot * 4 + (size_t)(RB_FIELDS + 4 * SCATTER_STEPS * DEFER_FIELDS) * (size_t)cap)));
    R *CK = ck.as<R>(), *SEG = seg.as<R>(), *YB = yb.as<R>(), *RS = rs.as<R>();
    const int64_t nn = MED == FGA_MEDIUM_GRID ? (int64_t)m->dev.n[0] * m->dev.n[1] * m->dev.n[2] : 0;
    ScopedDevBuf sgp, sgs;
    GradAcc<R> accp, accs;
    FGA_TRY(AccSetup<R>::make(grad_p, nn, sgp, s, accp));
    FGA_TRY(AccSetup<R>::make(grad_s, nn, sgs, s, accs));
    const R *ub = static_cast<const R *>(ubar);
    FGA_CUDA(cudaMemsetAsync(YB, 0, sizeof(R) * (size_t)slot, s));
    FGA_CUDA(cudaMemcpyAsync(CK, b->state.p, sizeof(R) * (size_t)slot, cudaMemcpyDeviceToDevice, s));
    const int32_t *fl = b->flags.as<int32_t>();
    const R dt = (R)sd->dt;
    // 1. checkpoints at steps C, 2C, ... (the last one at N when C does not divide N is not needed)
    NvtxRange nr_fwd("fga_solve_vjp: checkpoints");
    for (int cls = 0; cls < 4; cls++) {
        const int64_t nc = b->n_cls[cls];
        if (!nc) continue;
        const R sg = (cls & 1) ? R(-1) : R(1);
        const unsigned blocks = (unsigned)((nc + 127) / 128);
        ProfScope ps(P_ADJ_FWD, s);
        if (cls < 2)
            adj_forward_kernel<R, 0, MED><<<blocks, 128, 0, s>>>(m->dev, CK, CK, cap, slot, fl, b->off_cls[cls], nc, sg,
                                                                dt, (nseg - 1) * C, C);
        else
            adj_forward_kernel<R, 1, MED><<<blocks, 128, 0, s>>>(m->dev, CK, CK, cap, slot, fl, b->off_cls[cls], nc, sg,
                                                                dt, (nseg - 1) * C, C);
    }
    FGA_CUDA(cudaGetLastError());
    const size_t smem_max = 200 * 1024;
    int j = (int)sstep.size() - 1;
    int jst = 0;  // reverse steps since the last scatter of node cotangents
    for (int sgi = nseg - 1; sgi >= 0; sgi--) {
        NvtxRange nr_seg("fga_solve_vjp: segment (recompute, reverse)");
        const int n0 = sgi * C, len = std::min(C, N - n0);
        // 2a. the segment's states: slot 0 = checkpoint, slots 1..len recomputed
        FGA_CUDA(cudaMemcpyAsync(SEG, CK + (size_t)sgi * slot, sizeof(R) * (size_t)slot, cudaMemcpyDeviceToDevice, s));
        for (int cls = 0; cls < 4; cls++) {
            const int64_t nc = b->n_cls[cls];
            if (!nc) continue;
            const R sg = (cls & 1) ? R(-1) : R(1);
            const unsigned blocks = (unsigned)((nc + 127) / 128);
            ProfScope ps(P_ADJ_FWD, s);
            if (cls < 2)
                adj_forward_kernel<R, 0, MED><<<blocks, 128, 0, s>>>(m->dev, SEG, SEG, cap, slot, fl, b->off_cls[cls],
                                                                    nc, sg, dt, len, 1);
            else
                adj_forward_kernel<R, 1, MED><<<blocks, 128, 0, s>>>(m->dev, SEG, SEG, cap, slot, fl, b->off_cls[cls],
                                                                    nc, sg, dt, len, 1);
        }
        FGA_CUDA(cudaGetLastError());
        // 2b. reverse steps
        for (int n = n0 + len - 1; n >= n0; n--) {
            StepSamples ss{};
            for (int d = 0; d < 3; d++) {
                ss.lo[d] = box_lo[d];
                ss.hi[d] = box_hi[d];
            }
            int jl = j;
            while (jl >= 0 && sstep[(size_t)jl] == n) jl--;
            ss.nsj = j - jl;
            FGA_CHECK(ss.nsj <= 4, "fga_solve_vjp: more than 4 sample times inside one step");   // checked on entry
            const int jfirst = jl + 1;
            for (int q = 0; q < ss.nsj; q++) {
                const double th = sth[(size_t)(jfirst + q)];
                ss.th[q] = (float)th;
                ss.thd[q] = th;
                if (th > 0.0 && th < 1.0) ss.need_d1 = 1;
            }
            j = jl;
            const size_t smem = ss.nsj > 0 ? sizeof(R) * (size_t)nrx * (3 + 6 * (size_t)ss.nsj) : 0;
            FGA_CHECK(smem <= smem_max, "fga_solve_vjp: receivers x samples per step exceed the shared-memory stage");
            const R *ubs = ss.nsj > 0 ? ub + (size_t)jfirst * nrx * 6 : ub;
            const R *Sn = SEG + (size_t)(n - n0) * slot, *Sn1 = SEG + (size_t)(n - n0 + 1) * slot;
            const bool scatter = jst == SCATTER_STEPS - 1 || n == 0;
            for (int cls = 0; cls < 4; cls++) {
                const int64_t nc = b->n_cls[cls];
                if (!nc) continue;
                if (cls < 2)
                    FGA_TRY((reverse_step<R, 0, MED>(m->dev, Sn, Sn1, YB, RS, cap, slot, fl, b->off_cls[cls], nc,
                                                     (cls & 1) ? R(-1) : R(1), dt, (R)b->w, (R)b->k, (R)(rw * rw),
                                                     (int)nrx, rxd.as<R>(), ubs, ss, smem, accp, jst, scatter, s)));
                else
                    FGA_TRY((reverse_step<R, 1, MED>(m->dev, Sn, Sn1, YB, RS, cap, slot, fl, b->off_cls[cls], nc,
                                                     (cls & 1) ? R(-1) : R(1), dt, (R)b->w, (R)b->k, (R)(rw * rw),
                                                     (int)nrx, rxd.as<R>(), ubs, ss, smem, accs, jst, scatter, s)));
            }
            FGA_CUDA(cudaGetLastError());
            jst = scatter ? 0 : jst + 1;
        }
    }
    // 3. initial-velocity term
    if (bg) {
        for (int cls = 0; cls < 4; cls++) {
            const int64_t nc = b->n_cls[cls];
            if (!nc) continue;
            const unsigned blocks = (unsigned)((nc + 127) / 128);
            ProfScope ps(P_ADJ_INIT, s);
            if (cls < 2)
                adj_init_kernel<R, 0, MED><<<blocks, 128, 0, s>>>(m->dev, CK, bg->state.as<R>(), YB, cap,
                                                                 b->off_cls[cls], nc, accp);
            else
                adj_init_kernel<R, 1, MED><<<blocks, 128, 0, s>>>(m->dev, CK, bg->state.as<R>(), YB, cap,
                                                                 b->off_cls[cls], nc, accs);
        }
        FGA_CUDA(cudaGetLastError());
    }
    FGA_TRY(AccSetup<R>::finish(sgp, grad_p, nn, s));
    FGA_TRY(AccSetup<R>::finish(sgs, grad_s, nn, s));
    if (prof_counting()) prof_add_beam_steps(b->nb * (int64_t)N);
    FGA_CUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" fga_status fga_solve_vjp(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd_in,
                                    const void *ubar, double *grad_p, double *grad_s, int checkpoint_every,
                                    fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(m && init && sd_in, "fga_solve_vjp: NULL argument");
    FGA_CHECK(!(init->psi_rel_min > 0), "fga_solve_vjp: beam selection (psi_rel_min > 0) is not differentiated");
    // receivers given as (r, theta, phi): a Cartesian copy
    fga_solve_desc sdc;
    ScopedDevBuf rx_cart, snap_cart;
    FGA_TRY(cartesian_desc(sd_in, sdc, rx_cart, snap_cart, s));
    const fga_solve_desc *sd = &sdc;
    const int kind = m->dev.kind;
    if (kind != FGA_MEDIUM_GRID && kind != FGA_MEDIUM_CONST) {
        set_error("fga_solve_vjp: only grid (and constant) media are supported");
        return FGA_ERR_UNSUPPORTED;
    }
    FGA_CHECK(sd->nsteps >= 1 && std::isfinite(sd->dt) && sd->dt > 0.0, "fga_solve_vjp: nsteps >= 1 and dt > 0");
    FGA_CHECK(sd->n_times >= 1 && sd->times, "fga_solve_vjp: sample times missing");
    FGA_CHECK(!sd->rx_lattice, "fga_solve_vjp: receivers must be given as points");
    FGA_CHECK(sd->n_rx >= 1 && sd->rx && ubar, "fga_solve_vjp: receivers or cotangent missing");
    FGA_CHECK(kind != FGA_MEDIUM_GRID || (grad_p && grad_s), "fga_solve_vjp: gradient outputs missing");
    const int C = checkpoint_every > 0 ? checkpoint_every : 20;
    const double T = sd->dt * sd->nsteps;
    std::vector<int> sstep((size_t)sd->n_times);
    std::vector<double> sth((size_t)sd->n_times);
    for (int j = 0; j < sd->n_times; j++) {
        const double t = sd->times[j];
        FGA_CHECK(std::isfinite(t) && t > 0 && t <= T * (1 + 1e-12), "fga_solve_vjp: sample times must lie in (0, nsteps*dt]");
        FGA_CHECK(j == 0 || t > sd->times[j - 1], "fga_solve_vjp: times must be increasing");
        const double u = t / sd->dt;
        int n = std::min((int)std::floor(u), sd->nsteps - 1);
        sstep[(size_t)j] = n;
        sth[(size_t)j] = u - n;
    }
    // limits of the reverse steps, checked before any work: at most 4 samples inside one step, and the
    // receivers with that many samples' cotangents within the shared-memory stage of the record kernel
    {
        int most = 0;
        for (size_t j0 = 0; j0 < sstep.size();) {
            size_t j1 = j0;
            while (j1 < sstep.size() && sstep[j1] == sstep[j0]) j1++;
            most = std::max(most, (int)(j1 - j0));
            j0 = j1;
        }
        FGA_CHECK(most <= 4, "fga_solve_vjp: more than 4 sample times inside one step");
        const size_t rb = init->precision == FGA_PREC_FP64 ? 8 : 4;
        FGA_CHECK(rb * (size_t)sd->n_rx * (3 + 6 * (size_t)most) <= (size_t)200 * 1024,
                  "fga_solve_vjp: receivers x samples per step exceed the shared-memory stage");
    }
    fga_beams *b = nullptr, *bg = nullptr;
    FGA_TRY(decompose_impl(m, init, &b, s));
    struct Guard {
        fga_beams *b, **bg;
        DevBuf zero;
        ~Guard() {
            fga_beams_destroy(b);
            if (*bg) fga_beams_destroy(*bg);
            zero.release();
        }
    } guard{b, &bg, {}};
    if (init->g) {
        // beams of (f, g) = (0, g): their amplitudes are the initial-velocity parts a_G
        const size_t ny = (size_t)init->ny[0] * init->ny[1] * init->ny[2];
        FGA_TRY(guard.zero.ensure(ny * 3 * 16));
        FGA_CUDA(cudaMemsetAsync(guard.zero.p, 0, ny * 3 * 16, s));
        fga_init_desc d2 = *init;
        d2.f = guard.zero.p;
        FGA_TRY(decompose_impl(m, &d2, &bg, s));
        FGA_CHECK(bg->cap == b->cap && bg->nb == b->nb, "fga_solve_vjp: internal beam layout mismatch");
    }
    if (b->precision == FGA_PREC_FP64) {
        if (kind == FGA_MEDIUM_GRID)
            return run_vjp<double, FGA_MEDIUM_GRID>(m, init, sd, b, bg, sstep, sth, ubar, grad_p, grad_s, C, s);
        return run_vjp<double, FGA_MEDIUM_CONST>(m, init, sd, b, bg, sstep, sth, ubar, grad_p, grad_s, C, s);
    }
    if (kind == FGA_MEDIUM_GRID)
        return run_vjp<float, FGA_MEDIUM_GRID>(m, init, sd, b, bg, sstep, sth, ubar, grad_p, grad_s, C, s);
    return run_vjp<float, FGA_MEDIUM_CONST>(m, init, sd, b, bg, sstep, sth, ubar, grad_p, grad_s, C, s);
}
