// A7: beams in a medium of homogeneous layers (Sec. 3.1) between parallel planes, concentric spheres or
// undulating surfaces.  Inside a layer grad c = 0, so a beam moves on a straight line; a step that crosses an
// interface is split at the crossing, where the beam is replaced by its reflected and transmitted P and
// S children (Snell's law, plane-wave continuity of displacement and traction, and the dzQ/dzP jump of
// Eq. Inter_DzQDzP; at a sphere all of it in the local tangent-normal frame of the crossing point), and
// every child finishes the step.  Children are appended to the beam arrays with an atomic counter; the
// parent's slot goes to its first child.
#include <cmath>

#include "fga_beam.cuh"
#include "gather.cuh"

namespace fga {

namespace {

struct Cd {
    double r, i;
};
__device__ __forceinline__ Cd cadd(Cd a, Cd b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ Cd csub2(Cd a, Cd b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ Cd cmulx(Cd a, Cd b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cd cscale(Cd a, double s) { return {a.r * s, a.i * s}; }
__device__ __forceinline__ Cd cdivx(Cd a, Cd b) {
    const double d = b.r * b.r + b.i * b.i;
    return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__device__ __forceinline__ double cabs2(Cd a) { return a.r * a.r + a.i * a.i; }

// Layer speed of a beam (bits 4-7 of its flags hold its layer).
template <typename R> __device__ __forceinline__ R layer_speed(const ModelDev &M, int wave, int lay) {
    return wave ? mp<R>(M.lcs[lay], M.flcs[lay]) : mp<R>(M.lcp[lay], M.flcp[lay]);
}

// dy/dt in a homogeneous layer (grad c = 0): Q' = sg c P^, P' = 0, dzQ' = sg (c/|P|) dzP (I - P^P^T),
// dzP' = 0, amplitudes a' = (1/2) tr(Z^-1 Z') a (no SV/SH coupling: P is constant).
template <typename R>
__device__ __forceinline__ void layer_rhs(R sg, R c, const R *y, R *f) {
    const R P[3] = {y[F_P], y[F_P + 1], y[F_P + 2]};
    const R ip = Real<R>::rsqrt_(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    const R Ph[3] = {P[0] * ip, P[1] * ip, P[2] * ip};
    const R cip = c * ip;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        f[F_Q + d] = sg * c * Ph[d];
        f[F_P + d] = R(0);
    }
    C2<R> Z[3][3], Zd[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        R vr = R(0), vi = R(0);
#pragma unroll
        for (int l = 0; l < 3; l++) {
            vr += y[F_DP + 2 * (3 * m + l)] * Ph[l];
            vi += y[F_DP + 2 * (3 * m + l) + 1] * Ph[l];
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int e = 2 * (3 * m + j);
            f[F_DQ + e] = sg * cip * (y[F_DP + e] - vr * Ph[j]);
            f[F_DQ + e + 1] = sg * cip * (y[F_DP + e + 1] - vi * Ph[j]);
            f[F_DP + e] = R(0);
            f[F_DP + e + 1] = R(0);
            Z[m][j] = {y[F_DQ + e] - y[F_DP + e + 1], y[F_DQ + e + 1] + y[F_DP + e]};
            Zd[m][j] = {f[F_DQ + e], f[F_DQ + e + 1]};
        }
    }
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
    const R gr = R(0.5) * (tr * dr + ti * di) * idn, gi = R(0.5) * (ti * dr - tr * di) * idn;
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const R ar = y[F_A0 + 2 * q], ai = y[F_A0 + 2 * q + 1];
        f[F_A0 + 2 * q] = gr * ar - gi * ai;
        f[F_A0 + 2 * q + 1] = gr * ai + gi * ar;
    }
}

// one classical RK4 step of size h: out = y + the step's increment (summed at its own scale), Q by
// compensated summation with the compensation qc carried in and out
template <typename R>
__device__ __forceinline__ void layer_rk4(R sg, R c, const R *y, R h, R *out, R *qc) {
    R k[NF], t[NF], inc[NF];
    layer_rhs<R>(sg, c, y, k);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        inc[f] = h / R(6) * k[f];
        t[f] = y[f] + R(0.5) * h * k[f];
    }
    layer_rhs<R>(sg, c, t, k);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        inc[f] += h / R(3) * k[f];
        t[f] = y[f] + R(0.5) * h * k[f];
    }
    layer_rhs<R>(sg, c, t, k);
#pragma unroll
    for (int f = 0; f < NF; f++) {
        inc[f] += h / R(3) * k[f];
        t[f] = y[f] + h * k[f];
    }
    layer_rhs<R>(sg, c, t, k);
#pragma unroll
    for (int f = 3; f < NF; f++) out[f] = y[f] + (inc[f] + h / R(6) * k[f]);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        R q = y[F_Q + d];
        kahan_add<R>(q, qc[d], inc[F_Q + d] + h / R(6) * k[F_Q + d]);
        out[F_Q + d] = q;
    }
}

// Solve the 6x6 complex system A x = b (partial pivoting); false if singular.
__device__ bool csolve6_dev(Cd A[6][6], Cd b[6], Cd x[6]) {
    for (int c = 0; c < 6; c++) {
        int piv = c;
        for (int r = c + 1; r < 6; r++)
            if (cabs2(A[r][c]) > cabs2(A[piv][c])) piv = r;
        if (cabs2(A[piv][c]) < 1e-300) return false;
        if (piv != c) {
            for (int j = 0; j < 6; j++) {
                const Cd t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
            const Cd t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < 6; r++) {
            const Cd f = cdivx(A[r][c], A[c][c]);
            for (int j = c; j < 6; j++) A[r][j] = csub2(A[r][j], cmulx(f, A[c][j]));
            b[r] = csub2(b[r], cmulx(f, b[c]));
        }
    }
    for (int r = 5; r >= 0; r--) {
        Cd s = b[r];
        for (int j = r + 1; j < 6; j++) s = csub2(s, cmulx(A[r][j], x[j]));
        x[r] = cdivx(s, A[r][r]);
    }
    return true;
}

// Child i of the event (0 reflected P, 1 reflected S, 2 transmitted P, 3 transmitted S), FP64.
struct EventOut {
    int n;
    int slot[4];
    double P[4][3];
    Cd a0[4], a1[4];  // P: a0; S: (a_sv, a_sh) in the child's own frame
    int flags[4];
    double kappa[4];
};

// The scattering at an interface between layer la (incident side) and lb.  y holds the incident
// state (its Q on the interface).  Polarisations: P along P/|P|; SH along nsh = e3 x P/|e3 x P|
// (common to all waves of the event; e2 at normal incidence); SV along nsh x P/|P|.  Unknown
// amplitudes (rP, rSV, rSH, tP, tSV, tSH) make displacement and traction sigma.e3 continuous.
template <typename R>
__device__ __noinline__ void interface_event(const ModelDev &M, int fl, const R *y, int lb, double rel_min,
                                             EventOut &ev) {
    const int la = (fl >> 4) & 15, cls = fl & FL_CLASS_MASK, wave = cls >= 2;
    const double sgn = (cls & 1) ? -1.0 : 1.0;
    const double P0 = (double)y[F_P], P1 = (double)y[F_P + 1], P2 = (double)y[F_P + 2];
    const double cin = wave ? M.lcs[la] : M.lcp[la];
    const double pin = sqrt(P0 * P0 + P1 * P1 + P2 * P2), om = cin * pin;
    const double ph2 = P0 * P0 + P1 * P1;
    double nsh[3] = {0.0, 1.0, 0.0};
    if (ph2 > 0.0) {
        const double phn = sqrt(ph2);
        nsh[0] = -P1 / phn;
        nsh[1] = P0 / phn;
    }
    // incident displacement
    Cd U[3];
    {
        const double Ph[3] = {P0 / pin, P1 / pin, P2 / pin};
        const Cd a0 = {(double)y[F_A0], (double)y[F_A0 + 1]};
        if (!wave) {
            for (int d = 0; d < 3; d++) U[d] = cscale(a0, Ph[d]);
        } else {
            const Cd a1 = {(double)y[F_A1], (double)y[F_A1 + 1]};
            double Pd[3] = {P0, P1, P2}, Nsv[3], Nsh[3];
            s_frame<double>(Pd, (fl & FL_REF_E1) != 0, Nsv, Nsh);
            for (int d = 0; d < 3; d++) U[d] = cadd(cscale(a0, Nsv[d]), cscale(a1, Nsh[d]));
        }
    }
    const double lam[2] = {M.lrho[la] * (M.lcp[la] * M.lcp[la] - 2.0 * M.lcs[la] * M.lcs[la]),
                           M.lrho[lb] * (M.lcp[lb] * M.lcp[lb] - 2.0 * M.lcs[lb] * M.lcs[lb])};
    const double mu[2] = {M.lrho[la] * M.lcs[la] * M.lcs[la], M.lrho[lb] * M.lcs[lb] * M.lcs[lb]};
    auto traction = [&](int side, const Cd P[3], const Cd N[3], Cd T[3]) {
        const Cd pn = cadd(cadd(cmulx(P[0], N[0]), cmulx(P[1], N[1])), cmulx(P[2], N[2]));
        for (int i = 0; i < 3; i++) T[i] = cscale(cadd(cmulx(P[i], N[2]), cmulx(P[2], N[i])), mu[side]);
        T[2] = cadd(T[2], cscale(pn, lam[side]));
    };
    Cd Tin[3];
    {
        const Cd Pc[3] = {{P0, 0.0}, {P1, 0.0}, {P2, 0.0}};
        traction(0, Pc, U, Tin);
    }
    const double sz = P2 >= 0.0 ? 1.0 : -1.0;
    Cd Pw[4][3];
    double pnw[4], cw[4];
    bool prop[4];
    for (int w = 0; w < 4; w++) {
        const int trans = w >= 2, sw = w & 1, L = trans ? lb : la;
        cw[w] = sw ? M.lcs[L] : M.lcp[L];
        pnw[w] = om / cw[w];
        const double pz2 = pnw[w] * pnw[w] - ph2, side = trans ? sz : -sz;
        Pw[w][0] = {P0, 0.0};
        Pw[w][1] = {P1, 0.0};
        if (pz2 >= 0.0) {
            Pw[w][2] = {side * sqrt(pz2), 0.0};
            prop[w] = true;
        } else {
            Pw[w][2] = {0.0, sgn * side * sqrt(-pz2)};  // decays away from the interface
            prop[w] = false;
        }
    }
    auto pol = [&](int w, int which, Cd N[3]) {
        if (which == 0) {
            for (int d = 0; d < 3; d++) N[d] = cscale(Pw[w][d], 1.0 / pnw[w]);
        } else if (which == 2) {
            for (int d = 0; d < 3; d++) N[d] = {nsh[d], 0.0};
        } else {
            const double ip = 1.0 / pnw[w];
            N[0] = cscale(csub2(cscale(Pw[w][2], nsh[1]), cscale(Pw[w][1], nsh[2])), ip);
            N[1] = cscale(csub2(cscale(Pw[w][0], nsh[2]), cscale(Pw[w][2], nsh[0])), ip);
            N[2] = cscale(csub2(cscale(Pw[w][1], nsh[0]), cscale(Pw[w][0], nsh[1])), ip);
        }
    };
    Cd A[6][6], b[6], x[6];
    const int wv[6] = {0, 1, 1, 2, 3, 3}, pl[6] = {0, 1, 2, 0, 1, 2};
    for (int u = 0; u < 6; u++) {
        const int w = wv[u], trans = w >= 2;
        Cd N[3], T[3];
        pol(w, pl[u], N);
        traction(trans, Pw[w], N, T);
        const double s = trans ? -1.0 : 1.0;
        for (int d = 0; d < 3; d++) {
            A[d][u] = cscale(N[d], s);
            A[3 + d][u] = cscale(T[d], s);
        }
    }
    for (int d = 0; d < 3; d++) {
        b[d] = cscale(U[d], -1.0);
        b[3 + d] = cscale(Tin[d], -1.0);
    }
    ev.n = 0;
    if (!csolve6_dev(A, b, x)) return;
    const double ain = sqrt(cabs2(U[0]) + cabs2(U[1]) + cabs2(U[2]));
    const int gen = (fl >> 8) & 15;
    for (int w = 0; w < 4; w++) {
        if (!prop[w]) continue;
        const int sw = w & 1, trans = w >= 2;
        const Cd a0 = sw ? x[w == 1 ? 1 : 4] : x[w == 0 ? 0 : 3];
        const Cd a1 = sw ? x[w == 1 ? 2 : 5] : Cd{0.0, 0.0};
        const double amag = sqrt(cabs2(a0) + cabs2(a1));
        if (!(amag >= rel_min * ain) || amag == 0.0) continue;
        const int k = ev.n++;
        ev.slot[k] = w;
        for (int d = 0; d < 3; d++) ev.P[k][d] = Pw[w][d].r;
        ev.kappa[k] = (cw[w] / cin) * (cw[w] / cin);
        int cc = (sw ? 2 : 0) | (cls & 1);
        int flc = cc | ((trans ? lb : la) << 4) | ((gen + 1) << 8) | (fl & (3 << FL_ROOT_SHIFT));
        if (!sw) {
            ev.a0[k] = a0;
            ev.a1[k] = {0.0, 0.0};
        } else {
            // global SV/SH vectors -> the child's own frame (e3 unless its P is near vertical)
            Cd Nsv[3];
            pol(w, 1, Nsv);
            Cd Ag[3];
            for (int d = 0; d < 3; d++) Ag[d] = cadd(cmulx(a0, Nsv[d]), cscale(a1, nsh[d]));
            double Pc[3] = {ev.P[k][0], ev.P[k][1], ev.P[k][2]};
            const bool r1 = (Pc[0] * Pc[0] + Pc[1] * Pc[1]) < 0.01 * (Pc[0] * Pc[0] + Pc[1] * Pc[1] + Pc[2] * Pc[2]);
            if (r1) flc |= FL_REF_E1;
            double fsv[3], fsh[3];
            s_frame<double>(Pc, r1, fsv, fsh);
            Cd s0 = {0.0, 0.0}, s1 = {0.0, 0.0};
            for (int d = 0; d < 3; d++) {
                s0 = cadd(s0, cscale(Ag[d], fsv[d]));
                s1 = cadd(s1, cscale(Ag[d], fsh[d]));
            }
            ev.a0[k] = s0;
            ev.a1[k] = s1;
        }
        ev.flags[k] = flc;
    }
}

// Write child k of the event into out[] (NF reals): Q at the crossing, new P, dzQ F, dzP F^{-T},
// amplitudes.
template <typename R>
__device__ void make_child(const R *yc, const EventOut &ev, int k, R *out) {
#pragma unroll
    for (int f = 0; f < NF; f++) out[f] = yc[f];
    const double pz_in = (double)yc[F_P + 2];
    const double f20 = (ev.kappa[k] - 1.0) * (double)yc[F_P] / pz_in;
    const double f21 = (ev.kappa[k] - 1.0) * (double)yc[F_P + 1] / pz_in;
    const double f22 = ev.kappa[k] * ev.P[k][2] / pz_in;
    // F = I except the last row (f20, f21, f22); F^{-T} = I except the last column (-f20/f22, -f21/f22, 1/f22)
    for (int m = 0; m < 3; m++) {
        for (int c = 0; c < 2; c++) {  // re, im
            const double q0 = yc[F_DQ + 2 * (3 * m) + c], q1 = yc[F_DQ + 2 * (3 * m + 1) + c],
                         q2 = yc[F_DQ + 2 * (3 * m + 2) + c];
            out[F_DQ + 2 * (3 * m) + c] = (R)(q0 + q2 * f20);
            out[F_DQ + 2 * (3 * m + 1) + c] = (R)(q1 + q2 * f21);
            out[F_DQ + 2 * (3 * m + 2) + c] = (R)(q2 * f22);
            const double p0 = yc[F_DP + 2 * (3 * m) + c], p1 = yc[F_DP + 2 * (3 * m + 1) + c],
                         p2 = yc[F_DP + 2 * (3 * m + 2) + c];
            out[F_DP + 2 * (3 * m) + c] = (R)p0;
            out[F_DP + 2 * (3 * m + 1) + c] = (R)p1;
            out[F_DP + 2 * (3 * m + 2) + c] = (R)((p2 - p0 * f20 - p1 * f21) / f22);
        }
    }
    for (int d = 0; d < 3; d++) out[F_P + d] = (R)ev.P[k][d];
    out[F_A0] = (R)ev.a0[k].r;
    out[F_A0 + 1] = (R)ev.a0[k].i;
    out[F_A1] = (R)ev.a1[k].r;
    out[F_A1 + 1] = (R)ev.a1[k].i;
}

// Spherical layers (interfaces |x - c| = rho_i, rho_i = -zif[i] decreasing): the first crossing of the
// straight path q0 -> q1 of one step (a beam moves on a line in a homogeneous layer) with a sphere that
// bounds layer L, s(th) = q0 - c + th d, d = q1 - q0, |s(th)|^2 = a th^2 + b th + |q0 - c|^2.  The inner
// sphere is met when the path heads inward (b < 0) and the smaller root, 2 c0 / (-b + sqrt D), lies below
// 1 (a path may dip into it and leave again within one step); the outer sphere bounds a convex ball, so
// only an end point beyond it means a crossing, at the positive root.  Returns false without a crossing,
// else the fraction th of the step, the layer lb entered and the radius crossed.
__device__ bool shell_crossing(const ModelDev &M, int L, const double q0[3], const double q1[3], double &th, int &lb,
                               double &rho) {
    double s0[3], d[3], s1[3];
    for (int c = 0; c < 3; c++) {
        s0[c] = q0[c] - M.ctr[c];
        s1[c] = q1[c] - M.ctr[c];
        d[c] = q1[c] - q0[c];
    }
    const double a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double b = 2.0 * (s0[0] * d[0] + s0[1] * d[1] + s0[2] * d[2]);
    const double ss = s0[0] * s0[0] + s0[1] * s0[1] + s0[2] * s0[2];
    bool hit = false;
    if (L < M.nlay - 1) {
        const double r = -M.zif[L];
        const double c0 = ss - r * r, D = b * b - 4.0 * a * c0;
        if (b < 0.0 && D >= 0.0) {
            const double t = 2.0 * c0 / (-b + sqrt(D));
            if (t < 1.0) {
                th = t;
                lb = L + 1;
                rho = r;
                hit = true;
            }
        }
    }
    if (L > 0) {
        const double r = -M.zif[L - 1];
        if (s1[0] * s1[0] + s1[1] * s1[1] + s1[2] * s1[2] > r * r) {
            const double c0 = ss - r * r, D = fmax(b * b - 4.0 * a * c0, 0.0);
            const double t = b <= 0.0 ? (-b + sqrt(D)) / (2.0 * a) : -2.0 * c0 / (b + sqrt(D));
            if (!hit || t < th) {
                th = t;
                lb = L - 1;
                rho = r;
                hit = true;
            }
        }
    }
    return hit;
}

// FP32 screen for spherical layers: true when the straight path q0 -> q1 certainly meets no sphere of
// layer L, i.e. the end point lies inside the enclosing sphere and the path's closest approach to the
// centre lies outside the inner one, each with a relative margin of 1e-5 on r^2.
__device__ __forceinline__ bool shell_clear(const ModelDev &M, int L, const float *q0, const float *q1) {
    const float c0 = (float)M.ctr[0], c1 = (float)M.ctr[1], c2 = (float)M.ctr[2];
    const float s0[3] = {q0[0] - c0, q0[1] - c1, q0[2] - c2};
    const float d[3] = {q1[0] - q0[0], q1[1] - q0[1], q1[2] - q0[2]};
    const float r0 = s0[0] * s0[0] + s0[1] * s0[1] + s0[2] * s0[2];
    const float a = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const float b = 2.0f * (s0[0] * d[0] + s0[1] * d[1] + s0[2] * d[2]);
    if (L > 0) {
        const float ro = M.fzif[L - 1];                      // minus the enclosing radius
        const float r1 = r0 + b + a;                         // |q1 - c|^2
        if (!(r1 < ro * ro * (1.0f - 1e-5f))) return false;
    }
    if (L < M.nlay - 1) {
        const float ri = M.fzif[L];
        float t = b < 0.0f ? -b / (2.0f * a) : 0.0f;         // closest approach on the path
        t = t > 1.0f ? 1.0f : t;
        const float rmin = r0 + t * (b + a * t);
        if (!(rmin > ri * ri * (1.0f + 1e-5f))) return false;
    }
    return true;
}
__device__ __forceinline__ bool shell_clear(const ModelDev &, int, const double *, const double *) { return false; }

// Undulating layers: height of interface i above (x1, x2), and its slopes dh/dx1, dh/dx2.
__device__ __forceinline__ double surf_h(const ModelDev &M, int i, double x1, double x2) {
    return M.zif[i] + M.uamp[i] * cos(M.uk[0] * x1) * cos(M.uk[1] * x2);
}
__device__ __forceinline__ void surf_grad(const ModelDev &M, int i, double x1, double x2, double &h1, double &h2) {
    double s1, c1, s2, c2;
    sincos(M.uk[0] * x1, &s1, &c1);
    sincos(M.uk[1] * x2, &s2, &c2);
    h1 = -M.uamp[i] * M.uk[0] * s1 * c2;
    h2 = -M.uamp[i] * M.uk[1] * c1 * s2;
}

// FP32 screen for undulating layers: true when the end point q1 lies clearly between the interfaces that
// bound layer L (by a margin far above the FP32 rounding of the heights, which grows with the phase
// k |x| of the cosines).
__device__ __forceinline__ bool surf_clear(const ModelDev &M, int L, const float *q1) {
    const float cc = cosf(M.fuk[0] * q1[0]) * cosf(M.fuk[1] * q1[1]);
    const float ph = M.fuk[0] * fabsf(q1[0]) + M.fuk[1] * fabsf(q1[1]);
    if (L < M.nlay - 1) {
        const float h = M.fzif[L] + M.fuamp[L] * cc;
        const float m = 1e-4f * (1.0f + fabsf(M.fzif[L]) + fabsf(M.fuamp[L])) + 2e-6f * fabsf(M.fuamp[L]) * ph;
        if (!(q1[2] < h - m)) return false;
    }
    if (L > 0) {
        const float h = M.fzif[L - 1] + M.fuamp[L - 1] * cc;
        const float m = 1e-4f * (1.0f + fabsf(M.fzif[L - 1]) + fabsf(M.fuamp[L - 1])) + 2e-6f * fabsf(M.fuamp[L - 1]) * ph;
        if (!(q1[2] >= h + m)) return false;
    }
    return true;
}
__device__ __forceinline__ bool surf_clear(const ModelDev &, int, const double *) { return false; }

// Undulating layers: the first crossing of the straight path q0 -> q1 of one step with an interface that
// bounds layer L.  An end point on or below the lower interface (above the upper one) means a crossing;
// g(th) = x3(th) - h(x1(th), x2(th)) then changes sign on [0, 1] and its root is found by Newton's method
// kept inside a shrinking bracket (bisection where a Newton step leaves it; at most 100 iterations).  A
// start already beyond the interface (no sign change) takes the root of g's linear interpolation (the start
// itself when g does not change along the path).
// Returns false without a crossing, else th, the layer lb entered and the interface index.
__device__ bool surf_crossing(const ModelDev &M, int L, const double q0[3], const double q1[3], double &th, int &lb,
                              int &iface) {
    const double d[3] = {q1[0] - q0[0], q1[1] - q0[1], q1[2] - q0[2]};
    bool hit = false;
    for (int side = 0; side < 2; side++) {
        const bool down = side == 0;
        const int i = down ? L : L - 1;
        if (i < 0 || i > M.nlay - 2) continue;
        const double g0 = q0[2] - surf_h(M, i, q0[0], q0[1]), g1 = q1[2] - surf_h(M, i, q1[0], q1[1]);
        if (down ? !(g1 >= 0.0) : !(g1 < 0.0)) continue;
        double t;
        if ((g0 < 0.0) == down) {
            double lo = 0.0, hi = 1.0, glo = g0;   // g(lo) and g(hi) of opposite signs
            t = g0 / (g0 - g1);
            for (int it = 0; it < 100 && hi - lo > 1e-15; it++) {
                const double x1 = q0[0] + t * d[0], x2 = q0[1] + t * d[1];
                const double g = q0[2] + t * d[2] - surf_h(M, i, x1, x2);
                if (g == 0.0) break;
                if ((g < 0.0) == (glo < 0.0)) {
                    lo = t;
                    glo = g;
                } else {
                    hi = t;
                }
                double h1, h2;
                surf_grad(M, i, x1, x2, h1, h2);
                const double dg = d[2] - h1 * d[0] - h2 * d[1];
                double tn = dg != 0.0 ? t - g / dg : 0.5 * (lo + hi);
                if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
                if (fabs(tn - t) < 1e-16) {
                    t = tn;
                    break;
                }
                t = tn;
            }
        } else {
            t = g0 != g1 ? g0 / (g0 - g1) : 0.0;   // no motion across the surface: the start itself
        }
        if (!hit || t < th) {
            th = t;
            lb = down ? L + 1 : L - 1;
            iface = i;
            hit = true;
        }
    }
    return hit;
}

}  // namespace

// Write child ce (with its Q compensation) of the beam in slot b: the first child takes the parent's slot,
// the others are appended (atomic counter); children beyond cap are counted in counts[1].
template <typename R>
__device__ void store_child(R *__restrict__ st, int32_t *__restrict__ flags, int32_t *__restrict__ ids,
                            long long *__restrict__ path, int64_t cap, unsigned long long *__restrict__ counts, int64_t b,
                            int k, const R *ce, const R *qch, int flc, int32_t id, long long pp, int slot) {
    int64_t dst = b;
    if (k > 0) {
        dst = (int64_t)atomicAdd(&counts[0], 1ull);
        if (dst >= cap) {
            atomicAdd(&counts[1], 1ull);
            return;
        }
    }
#pragma unroll
    for (int f = 0; f < NF; f++) st[(int64_t)f * cap + dst] = ce[f];
#pragma unroll
    for (int d = 0; d < 3; d++) st[(int64_t)(F_QC + d) * cap + dst] = qch[d];
    flags[dst] = flc;
    ids[dst] = id;
    path[dst] = pp * 4 + slot + 1;
}

// The interface event of beam b in curved layers (SHAPE 1: spheres, SHAPE 2: undulating interfaces), at
// fraction th of the step where it enters layer lb through the sphere of radius rho or through interface
// iface.  The beam (still unchanged in st) advances to the crossing, which is put on the interface in FP64
// (radially onto the sphere, vertically onto the undulating surface; its FP32 rounding goes to the Q
// compensation), and is rotated into the local frame whose third axis is the interface's normal there; the
// flat-interface event runs in that frame (Sec. 3.1: the tangent plane stands in for the interface), and
// every child is rotated back and finishes the step.  Kept out of line and reading its beam from memory, so
// that the step kernel's state stays in registers.
template <typename R, int SHAPE>
__device__ __noinline__ void curved_event_step(const ModelDev &M, R *__restrict__ st, int32_t *__restrict__ flags,
                                               int32_t *__restrict__ ids, long long *__restrict__ path, int64_t cap,
                                               unsigned long long *__restrict__ counts, R dt, double rel_min, int64_t b,
                                               int fl, R sg, R c, double th, int lb, double rho, int iface) {
    R y[NF], yc[NF], qc[3];
    for (int f = 0; f < NF; f++) y[f] = st[(int64_t)f * cap + b];
    for (int d = 0; d < 3; d++) qc[d] = st[(int64_t)(F_QC + d) * cap + b];
    layer_rk4<R>(sg, c, y, (R)th * dt, yc, qc);
    double x[3], nrm[3], Rl[9];
    for (int d = 0; d < 3; d++) x[d] = (double)yc[F_Q + d] - (double)qc[d];
    if (SHAPE == 1) {
        double s[3], sn = 0.0;
        for (int d = 0; d < 3; d++) {
            s[d] = x[d] - M.ctr[d];
            sn += s[d] * s[d];
        }
        sn = sqrt(sn);
        for (int d = 0; d < 3; d++) {
            nrm[d] = s[d] / sn;
            x[d] = M.ctr[d] + rho * nrm[d];
        }
    } else {
        x[2] = surf_h(M, iface, x[0], x[1]);
        double h1, h2;
        surf_grad(M, iface, x[0], x[1], h1, h2);
        const double nn = sqrt(1.0 + h1 * h1 + h2 * h2);
        nrm[0] = -h1 / nn;
        nrm[1] = -h2 / nn;
        nrm[2] = 1.0 / nn;
    }
    for (int d = 0; d < 3; d++) {
        yc[F_Q + d] = (R)x[d];
        qc[d] = (R)((double)yc[F_Q + d] - x[d]);
    }
    frame_from_normal(nrm, Rl);
    int fll = fl;
    rotate_state<R>(Rl, false, false, yc, fll);   // Q stays global: the event does not read it
    EventOut ev;
    interface_event<R>(M, fll, yc, lb, rel_min, ev);
    if (ev.n == 0) {
        flags[b] = fl | FL_DEAD;
        return;
    }
    const long long pp = path[b];
    const int32_t id = ids[b];
    for (int k = 0; k < ev.n; k++) {
        R ch[NF], ce[NF], qch[3] = {qc[0], qc[1], qc[2]};
        make_child<R>(yc, ev, k, ch);
        int flc = ev.flags[k];
        rotate_state<R>(Rl, true, false, ch, flc);
        const R sgc = (flc & 1) ? R(-1) : R(1);
        layer_rk4<R>(sgc, layer_speed<R>(M, (flc & FL_CLASS_MASK) >= 2, (flc >> 4) & 15), ch, R(1.0 - th) * dt, ce,
                     qch);
        store_child<R>(st, flags, ids, path, cap, counts, b, k, ce, qch, flc, id, pp, ev.slot[k]);
    }
}

// One step for every beam alive at the start of the step (n_begin = *counts); children beyond the
// first are appended at *counts (atomic); overflow beyond cap is counted in counts[1].
template <typename R, int SHAPE>
__global__ void __launch_bounds__(128) layered_step_kernel(ModelDev M, R *__restrict__ st, int32_t *__restrict__ flags,
                                                          int32_t *__restrict__ ids, long long *__restrict__ path,
                                                          int64_t cap, const int64_t *__restrict__ n_begin,
                                                          unsigned long long *__restrict__ counts, R dt, int gmax,
                                                          double rel_min) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= *n_begin) return;
    const int fl = flags[b];
    if (fl & FL_DEAD) return;
    const int wave = (fl & FL_CLASS_MASK) >= 2, L = (fl >> 4) & 15;
    const R sg = (fl & 1) ? R(-1) : R(1);
    R y[NF], y1[NF], qc[3], qc1[3];
#pragma unroll
    for (int f = 0; f < NF; f++) y[f] = st[(int64_t)f * cap + b];
#pragma unroll
    for (int d = 0; d < 3; d++) qc1[d] = qc[d] = st[(int64_t)(F_QC + d) * cap + b];
    const R c = layer_speed<R>(M, wave, L);
    layer_rk4<R>(sg, c, y, dt, y1, qc1);
    if (SHAPE != 0) {
        // FP32: a step that stays clear of the interfaces of its layer (by a margin far above the rounding of
        // the screen) is decided by the screen; the rest take the exact FP64 test
        bool hit = false;
        double th = 0.0, rho = 0.0;
        int lb = L, iface = 0;
        const bool clear = sizeof(R) == 4 && (SHAPE == 1 ? shell_clear(M, L, y + F_Q, y1 + F_Q)
                                                          : surf_clear(M, L, y1 + F_Q));
        if (!clear) {
            double q0[3], q1[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                q0[d] = (double)y[F_Q + d] - (double)qc[d];
                q1[d] = (double)y1[F_Q + d] - (double)qc1[d];
            }
            hit = SHAPE == 1 ? shell_crossing(M, L, q0, q1, th, lb, rho) : surf_crossing(M, L, q0, q1, th, lb, iface);
        }
        if (!hit) {
#pragma unroll
            for (int f = 0; f < NF; f++) st[(int64_t)f * cap + b] = y1[f];
#pragma unroll
            for (int d = 0; d < 3; d++) st[(int64_t)(F_QC + d) * cap + b] = qc1[d];
        } else if (((fl >> 8) & 15) >= gmax) {
            flags[b] = fl | FL_DEAD;
        } else {
            curved_event_step<R, SHAPE>(M, st, flags, ids, path, cap, counts, dt, rel_min, b, fl, sg, c, th, lb, rho,
                                        iface);
        }
        return;
    }
    const R ztop = L > 0 ? mp<R>(M.zif[L - 1], M.fzif[L - 1]) : -R(INFINITY);
    const R zbot = L < M.nlay - 1 ? mp<R>(M.zif[L], M.fzif[L]) : R(INFINITY);
    if (y1[F_Q + 2] >= ztop && y1[F_Q + 2] < zbot) {
#pragma unroll
        for (int f = 0; f < NF; f++) st[(int64_t)f * cap + b] = y1[f];
#pragma unroll
        for (int d = 0; d < 3; d++) st[(int64_t)(F_QC + d) * cap + b] = qc1[d];
        return;
    }
    // the step crosses an interface: advance to it, scatter, finish the step with every child
    const bool down = y1[F_Q + 2] >= zbot;
    const R zc = down ? zbot : ztop;
    const int lb = down ? L + 1 : L - 1;
    const R th = (zc - y[F_Q + 2]) / (y1[F_Q + 2] - y[F_Q + 2]);
    if (((fl >> 8) & 15) >= gmax) {
        flags[b] = fl | FL_DEAD;
        return;
    }
    R yc[NF];
    layer_rk4<R>(sg, c, y, th * dt, yc, qc);
    yc[F_Q + 2] = zc;
    qc[2] = R(0);                 // the interface depth is exact
    EventOut ev;
    interface_event<R>(M, fl, yc, lb, rel_min, ev);
    if (ev.n == 0) {
        flags[b] = fl | FL_DEAD;
        return;
    }
    const long long pp = path[b];
    const int32_t id = ids[b];
    for (int k = 0; k < ev.n; k++) {
        R ch[NF], ce[NF], qch[3] = {qc[0], qc[1], qc[2]};
        make_child<R>(yc, ev, k, ch);
        const int flc = ev.flags[k];
        const R sgc = (flc & 1) ? R(-1) : R(1);
        layer_rk4<R>(sgc, layer_speed<R>(M, (flc & FL_CLASS_MASK) >= 2, (flc >> 4) & 15), ch, (R(1) - th) * dt, ce,
                     qch);
        store_child<R>(st, flags, ids, path, cap, counts, b, k, ce, qch, flc, id, pp, ev.slot[k]);
    }
}

__global__ void copy_count_kernel(const unsigned long long *counts, int64_t *n_begin, int64_t cap) {
    const unsigned long long n = counts[0];
    *n_begin = (int64_t)(n < (unsigned long long)cap ? n : (unsigned long long)cap);
}

fga_status launch_layered_steps(const fga_model *m, fga_beams *b, double dt, int nsteps, cudaStream_t s) {
    if (nsteps <= 0) return FGA_OK;
    const int T = 128;
    const unsigned blocks = (unsigned)((b->cap + T - 1) / T);
    for (int n = 0; n < nsteps; n++) {
        {
            ProfScope ps(P_OTHER_LAYER, s);
            copy_count_kernel<<<1, 1, 0, s>>>(b->counts.as<unsigned long long>(), b->n_begin.as<int64_t>(), b->cap);
        }
        prof_add_beam_steps(b->nb);
        ProfScope ps(P_PROP, s);
        // curved layers in their own instantiations, so that the planar kernel carries none of their code
        auto kd = m->dev.shells ? layered_step_kernel<double, 1>
                                : (m->dev.undul ? layered_step_kernel<double, 2> : layered_step_kernel<double, 0>);
        auto kf = m->dev.shells ? layered_step_kernel<float, 1>
                                : (m->dev.undul ? layered_step_kernel<float, 2> : layered_step_kernel<float, 0>);
        if (b->precision == FGA_PREC_FP64)
            kd<<<blocks, T, 0, s>>>(m->dev, b->state.as<double>(), b->flags.as<int32_t>(), b->id.as<int32_t>(),
                                    b->path.as<long long>(), b->cap, b->n_begin.as<int64_t>(),
                                    b->counts.as<unsigned long long>(), dt, b->gmax, b->rel_min);
        else
            kf<<<blocks, T, 0, s>>>(m->dev, b->state.as<float>(), b->flags.as<int32_t>(), b->id.as<int32_t>(),
                                    b->path.as<long long>(), b->cap, b->n_begin.as<int64_t>(),
                                    b->counts.as<unsigned long long>(), (float)dt, b->gmax, b->rel_min);
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

}  // namespace fga
