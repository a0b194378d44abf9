/*
 * fga_oracle.c -- plain FP64 CPU oracle of the frozen Gaussian approximation (FGA)
 * for the 3-D isotropic elastic wave equation (Hateley, Chai, Tong & Yang,
 * "Frozen Gaussian approximation for 3-D elastic wave equation and seismic
 * tomography", arXiv:1810.06760).
 *
 * THIS FILE IS TEST INFRASTRUCTURE. It exists to check the GPU library; it is
 * not part of the product path.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every routine follows the paper's equations step by step, in FP64, with no
 * blocking, fusion or reordering beyond what the equations state:
 *   - model sampling c, grad c, Hessian c                      (Sec. 2.2, Eqs. char_plus, DzDt)
 *   - wave-packet (FBI) transform, direct and separable         (Eqs. psi, alpha^k)
 *   - beam initialisation                                      (Eqs. FGA, ini_plus, amp_P..amp_SH, op_zZ_app)
 *   - right-hand side of the ray, Jacobian and amplitude ODEs   (Eqs. char_plus, char_minus, amp_P, amp_SV, amp_SH, DzDt)
 *   - classical RK4 with a fixed step                          (Sec. 2.3)
 *   - Gaussian summation, untruncated and truncated            (Eq. FGA)
 *   - cell binning of beam centres                             (no counterpart in the paper: the
 *                                                               fast summation it cites is not printed)
 *   - flat-interface Snell / Zoeppritz / F-W jump              (Sec. 3.1, Eqs. p:int, Yilmaz, Inter_DzQDzP)
 *
 * Readings of points the paper leaves open (each listed in the design doc):
 *   alpha uses |p| (not |p|^3) and c(q); S beams carry psi folded into (a_sv, a_sh);
 *   no phase S (it is identically zero for H = +-c|P|); the SV/SH frame is
 *   N_sh = e_ref x P / |e_ref x P|, N_sv = N_sh x P/|P| with e_ref = e3, or e1 for
 *   beams whose initial p lies within ~5.7 degrees of the vertical.
 *
 * Conventions: complex numbers are C99 double complex (re, im interleaved);
 * (DQ)_{mj} = dQ_j/dz_m is stored row-major DQ[3*m + j], same for DP.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ------------------------------------------------------------------------- */
/* velocity model                                                             */
/* ------------------------------------------------------------------------- */

enum { ORC_CONST = 0, ORC_SINE = 1, ORC_GRID = 2, ORC_LAYERED = 3 };

typedef struct {
    int kind;
    double cp0, cs0;        /* constant speeds; background of the sine medium */
    double amp;             /* sine medium: c_p = cp0 + amp sin(2 pi x1) sin(2 pi x2) sin(2 pi x3) */
    double cs_ratio;        /* sine medium: c_s = cs_ratio * c_p */
    int n[3];               /* grid medium: nodes per axis */
    double o[3], h[3];      /* grid medium: node (i,j,l) sits at o + (i h0, j h1, l h2) */
    const float *gp, *gs;   /* grid medium: 10 fields per node, node-major, axis 0 slowest */
    int nlay;               /* layered medium: nlay layers, nlay-1 interfaces zif (depth = x3, increasing) */
    const double *zif, *lcp, *lcs, *lrho;
} orc_model;

/* The 10 model fields at a point: c, dc/dx1..3, d2c/dx1dx1, dx1dx2, dx1dx3, dx2dx2, dx2dx3, dx3dx3. */

static void sine_fields(double c0, double A, double x1, double x2, double x3, double out[10])
{
    const double w = 2.0 * M_PI;
    double s1 = sin(w * x1), s2 = sin(w * x2), s3 = sin(w * x3);
    double k1 = cos(w * x1), k2 = cos(w * x2), k3 = cos(w * x3);
    out[0] = c0 + A * s1 * s2 * s3;
    out[1] = A * w * k1 * s2 * s3;
    out[2] = A * w * s1 * k2 * s3;
    out[3] = A * w * s1 * s2 * k3;
    out[4] = -A * w * w * s1 * s2 * s3;
    out[5] = A * w * w * k1 * k2 * s3;
    out[6] = A * w * w * k1 * s2 * k3;
    out[7] = -A * w * w * s1 * s2 * s3;
    out[8] = A * w * w * s1 * k2 * k3;
    out[9] = -A * w * w * s1 * s2 * s3;
}

/* Trilinear interpolation of all 10 node fields; positions outside the box are
 * clamped onto it (constant extension of every field). */
static void grid_fields(const orc_model *m, const float *g, const double x[3], double out[10])
{
    int i[3];
    double fr[3];
    for (int d = 0; d < 3; d++) {
        double t = (x[d] - m->o[d]) / m->h[d];
        if (t < 0.0) t = 0.0;
        if (t > (double)(m->n[d] - 1)) t = (double)(m->n[d] - 1);
        int id = (int)floor(t);
        if (id > m->n[d] - 2) id = m->n[d] - 2;
        i[d] = id;
        fr[d] = t - (double)id;
    }
    for (int f = 0; f < 10; f++) out[f] = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) {
                double wgt = (a ? fr[0] : 1.0 - fr[0]) * (b ? fr[1] : 1.0 - fr[1]) * (c ? fr[2] : 1.0 - fr[2]);
                size_t node = ((size_t)(i[0] + a) * m->n[1] + (size_t)(i[1] + b)) * m->n[2] + (size_t)(i[2] + c);
                for (int f = 0; f < 10; f++) out[f] += wgt * (double)g[node * 10 + f];
            }
}

static int layer_of(const orc_model *m, double z)
{
    int l = 0;
    while (l < m->nlay - 1 && z >= m->zif[l]) l++;
    return l;
}

/* wave = 0: P speed, wave = 1: S speed. */
void orc_model_eval(const orc_model *m, int wave, const double x[3], double out[10])
{
    switch (m->kind) {
    case ORC_CONST:
        for (int f = 0; f < 10; f++) out[f] = 0.0;
        out[0] = wave ? m->cs0 : m->cp0;
        break;
    case ORC_SINE:
        sine_fields(m->cp0, m->amp, x[0], x[1], x[2], out);
        if (wave)
            for (int f = 0; f < 10; f++) out[f] *= m->cs_ratio;
        break;
    case ORC_GRID:
        grid_fields(m, wave ? m->gs : m->gp, x, out);
        break;
    case ORC_LAYERED: {
        int l = layer_of(m, x[2]);
        for (int f = 0; f < 10; f++) out[f] = 0.0;
        out[0] = wave ? m->lcs[l] : m->lcp[l];
        break;
    }
    default:
        for (int f = 0; f < 10; f++) out[f] = 0.0;
    }
}

void orc_model_eval_many(const orc_model *m, int wave, int n, const double *x, double *out)
{
    for (int i = 0; i < n; i++) orc_model_eval(m, wave, x + 3 * i, out + 10 * i);
}

/* ------------------------------------------------------------------------- */
/* wave-packet (FBI) transform, Eq. psi                                       */
/* ------------------------------------------------------------------------- */
/* F(q,p) = sum_y f(y) exp(-i k p.(y-q) - k|y-q|^2/2) dy^3 on the y-grid
 * y_{d,i} = y0[d] + i dy[d].  Mesh points: q_{d,i} = q0[d] + i dq[d] (nq per
 * axis), p_{d,j} = p0[d] + j dp[d] (np per axis); mesh index
 * m = ((iq0 nq + iq1) nq + iq2) np^3 + (jp0 np + jp1) np + jp2.
 * f is complex [ny0][ny1][ny2][3]; F is complex [M][3]. */

void orc_fbi_direct(const int ny[3], const double y0[3], const double dy[3], const double *f_,
                    double k, int nq, const double q0[3], const double dq[3],
                    int np, const double p0[3], const double dp[3], double *F_)
{
    const cplx *f = (const cplx *)f_;
    cplx *F = (cplx *)F_;
    const long NP = (long)np * np * np;
    const long M = (long)nq * nq * nq * NP;
    const double vol = dy[0] * dy[1] * dy[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (long mi = 0; mi < M; mi++) {
        long iq = mi / NP, ip = mi % NP;
        int qi[3] = {(int)(iq / ((long)nq * nq)), (int)((iq / nq) % nq), (int)(iq % nq)};
        int pj[3] = {(int)(ip / ((long)np * np)), (int)((ip / np) % np), (int)(ip % np)};
        double q[3], p[3];
        for (int d = 0; d < 3; d++) {
            q[d] = q0[d] + qi[d] * dq[d];
            p[d] = p0[d] + pj[d] * dp[d];
        }
        cplx acc[3] = {0, 0, 0};
        for (int a = 0; a < ny[0]; a++)
            for (int b = 0; b < ny[1]; b++)
                for (int c = 0; c < ny[2]; c++) {
                    double y[3] = {y0[0] + a * dy[0], y0[1] + b * dy[1], y0[2] + c * dy[2]};
                    double pd = 0.0, r2 = 0.0;
                    for (int d = 0; d < 3; d++) {
                        pd += p[d] * (y[d] - q[d]);
                        r2 += (y[d] - q[d]) * (y[d] - q[d]);
                    }
                    cplx kern = cexp(-I * k * pd - 0.5 * k * r2);
                    const cplx *fy = f + (((size_t)a * ny[1] + b) * ny[2] + c) * 3;
                    for (int comp = 0; comp < 3; comp++) acc[comp] += fy[comp] * kern;
                }
        for (int comp = 0; comp < 3; comp++) F[mi * 3 + comp] = acc[comp] * vol;
    }
}

/* The same sum using that the kernel factors over the three axes:
 * exp(...) = prod_d K_d(q_d, p_d; y_d), K(q,p;y) = exp(-i k p (y-q) - k (y-q)^2 / 2).
 * Three contractions, one per axis, over the per-axis pair index a = iq*np + jp. */
void orc_fbi_separable(const int ny[3], const double y0[3], const double dy[3], const double *f_,
                       double k, int nq, const double q0[3], const double dq[3],
                       int np, const double p0[3], const double dp[3], double *F_)
{
    const cplx *f = (const cplx *)f_;
    cplx *F = (cplx *)F_;
    const int A = nq * np;
    cplx *K[3];
    for (int d = 0; d < 3; d++) {
        K[d] = (cplx *)malloc(sizeof(cplx) * A * ny[d]);
        for (int iq = 0; iq < nq; iq++)
            for (int jp = 0; jp < np; jp++) {
                double q = q0[d] + iq * dq[d], p = p0[d] + jp * dp[d];
                for (int i = 0; i < ny[d]; i++) {
                    double y = y0[d] + i * dy[d];
                    K[d][(size_t)(iq * np + jp) * ny[d] + i] = cexp(-I * k * p * (y - q) - 0.5 * k * (y - q) * (y - q));
                }
            }
    }
    /* stage 1: contract y2 */
    cplx *T1 = (cplx *)calloc((size_t)ny[0] * ny[1] * A * 3, sizeof(cplx));
#pragma omp parallel for collapse(2)
    for (int a = 0; a < ny[0]; a++)
        for (int b = 0; b < ny[1]; b++)
            for (int a2 = 0; a2 < A; a2++)
                for (int comp = 0; comp < 3; comp++) {
                    cplx s = 0;
                    for (int c = 0; c < ny[2]; c++)
                        s += f[(((size_t)a * ny[1] + b) * ny[2] + c) * 3 + comp] * K[2][(size_t)a2 * ny[2] + c];
                    T1[(((size_t)a * ny[1] + b) * A + a2) * 3 + comp] = s;
                }
    /* stage 2: contract y1 */
    cplx *T2 = (cplx *)calloc((size_t)ny[0] * A * A * 3, sizeof(cplx));
#pragma omp parallel for collapse(2)
    for (int a = 0; a < ny[0]; a++)
        for (int a1 = 0; a1 < A; a1++)
            for (int a2 = 0; a2 < A; a2++)
                for (int comp = 0; comp < 3; comp++) {
                    cplx s = 0;
                    for (int b = 0; b < ny[1]; b++)
                        s += T1[(((size_t)a * ny[1] + b) * A + a2) * 3 + comp] * K[1][(size_t)a1 * ny[1] + b];
                    T2[(((size_t)a * A + a1) * A + a2) * 3 + comp] = s;
                }
    /* stage 3: contract y0, then scatter (a0,a1,a2) -> mesh index */
    const double vol = dy[0] * dy[1] * dy[2];
    const long NP = (long)np * np * np;
#pragma omp parallel for collapse(2)
    for (int a0 = 0; a0 < A; a0++)
        for (int a1 = 0; a1 < A; a1++)
            for (int a2 = 0; a2 < A; a2++) {
                int iq0 = a0 / np, jp0 = a0 % np, iq1 = a1 / np, jp1 = a1 % np, iq2 = a2 / np, jp2 = a2 % np;
                long mi = (((long)iq0 * nq + iq1) * nq + iq2) * NP + ((long)jp0 * np + jp1) * np + jp2;
                for (int comp = 0; comp < 3; comp++) {
                    cplx s = 0;
                    for (int a = 0; a < ny[0]; a++)
                        s += T2[(((size_t)a * A + a1) * A + a2) * 3 + comp] * K[0][(size_t)a0 * ny[0] + a];
                    F[mi * 3 + comp] = s * vol;
                }
            }
    free(T1);
    free(T2);
    for (int d = 0; d < 3; d++) free(K[d]);
}

/* ------------------------------------------------------------------------- */
/* beam state                                                                  */
/* ------------------------------------------------------------------------- */

typedef struct {
    double Q[3], P[3];
    cplx DQ[9], DP[9];  /* dQ_j/dz_m at [3m+j]; dP_j/dz_m at [3m+j] */
    cplx a[3];          /* P: a[0]; S frame form: a[0]=a_sv, a[1]=a_sh; S vector form: polarised amplitude A */
} orc_state;            /* 48 doubles */

/* meta bits: 0-1 class (0 P+, 1 P-, 2 S+, 3 S-), bit 2: S frame reference e1 (else e3),
 * bit 3: S amplitude carried as a complex 3-vector (parallel-transport form) */
#define META_CLS(mt) ((mt) & 3)
#define META_REF_E1 4
#define META_VECTOR 8

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* S polarisation frame of a beam with propagation vector P. */
static void s_frame(const double P[3], int ref_e1, double Nsv[3], double Nsh[3], double *vnorm)
{
    double e[3] = {ref_e1 ? 1.0 : 0.0, 0.0, ref_e1 ? 0.0 : 1.0};
    double v[3], Ph[3];
    cross3(e, P, v);
    double nv = norm3(v), nP = norm3(P);
    for (int d = 0; d < 3; d++) {
        Nsh[d] = v[d] / nv;
        Ph[d] = P[d] / nP;
    }
    cross3(Nsh, Ph, Nsv);
    if (vnorm) *vnorm = nv;
}

/* The S frame reference axis is fixed per beam from its initial p: e3 unless p is
 * within asin(0.1) of the vertical. */
int orc_s_ref_e1(const double p[3])
{
    return (p[0] * p[0] + p[1] * p[1]) < 0.01 * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
}

/* Beam initialisation (Eqs. FGA, psi, alpha^k with |p| in the denominator, ini_plus/ini_minus,
 * op_zZ_app): Q = q, P = p, dzQ = I, dzP = -iI (so Z = 2I), amplitude 2^{3/2} times the weight
 * psi_pm = (F.n +- i G.n / (k c(q) |p|)) / 2, n the class's initial polarisation. */
void orc_beam_init(const orc_model *m, double k, int nq, const double q0[3], const double dq[3],
                   int np, const double p0[3], const double dp[3],
                   const double *F_, const double *G_, int cls, int vector_form,
                   double *st_, int *meta)
{
    const cplx *F = (const cplx *)F_;
    const cplx *G = (const cplx *)G_;
    orc_state *st = (orc_state *)st_;
    const long NP = (long)np * np * np;
    const long M = (long)nq * nq * nq * NP;
    const int wave = cls >= 2;
    const double sgn = (cls & 1) ? -1.0 : 1.0;
    for (long mi = 0; mi < M; mi++) {
        long iq = mi / NP, ip = mi % NP;
        int qi[3] = {(int)(iq / ((long)nq * nq)), (int)((iq / nq) % nq), (int)(iq % nq)};
        int pj[3] = {(int)(ip / ((long)np * np)), (int)((ip / np) % np), (int)(ip % np)};
        orc_state *y = st + mi;
        memset(y, 0, sizeof(*y));
        for (int d = 0; d < 3; d++) {
            y->Q[d] = q0[d] + qi[d] * dq[d];
            y->P[d] = p0[d] + pj[d] * dp[d];
        }
        for (int d = 0; d < 3; d++) {
            y->DQ[4 * d] = 1.0;
            y->DP[4 * d] = -I;
        }
        double cf[10];
        orc_model_eval(m, wave, y->Q, cf);
        double pn = norm3(y->P);
        const cplx *Fm = F + mi * 3;
        const cplx *Gm = G ? G + mi * 3 : NULL;
        double dirs[2][3];
        int ndir;
        int mt = cls;
        if (!wave) {
            for (int d = 0; d < 3; d++) dirs[0][d] = y->P[d] / pn;
            ndir = 1;
        } else {
            int r = orc_s_ref_e1(y->P);
            if (r) mt |= META_REF_E1;
            s_frame(y->P, r, dirs[0], dirs[1], NULL);
            ndir = 2;
        }
        cplx psi[2];
        for (int j = 0; j < ndir; j++) {
            cplx fn = 0, gn = 0;
            for (int d = 0; d < 3; d++) {
                fn += Fm[d] * dirs[j][d];
                if (Gm) gn += Gm[d] * dirs[j][d];
            }
            psi[j] = 0.5 * (fn + sgn * I * gn / (k * cf[0] * pn));
        }
        const double a0 = pow(2.0, 1.5);
        if (!wave) {
            y->a[0] = a0 * psi[0];
        } else if (!vector_form) {
            y->a[0] = a0 * psi[0];
            y->a[1] = a0 * psi[1];
        } else {
            mt |= META_VECTOR;
            for (int d = 0; d < 3; d++) y->a[d] = a0 * (psi[0] * dirs[0][d] + psi[1] * dirs[1][d]);
        }
        meta[mi] = mt;
    }
}

/* ------------------------------------------------------------------------- */
/* right-hand side of the beam ODEs                                           */
/* ------------------------------------------------------------------------- */

/* trace(Z^{-1} Zd) for complex 3x3 Z (invertible: Z Z^* = (Jv)^*(Jv) + 2I, App. A),
 * by Gauss-Jordan elimination with partial pivoting on [Z | Zd]. */
static cplx trace_solve(const cplx Z[9], const cplx Zd[9])
{
    cplx a[3][6];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            a[r][c] = Z[3 * r + c];
            a[r][3 + c] = Zd[3 * r + c];
        }
    for (int col = 0; col < 3; col++) {
        int piv = col;
        for (int r = col + 1; r < 3; r++)
            if (cabs(a[r][col]) > cabs(a[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 6; c++) {
                cplx t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        cplx inv = 1.0 / a[col][col];
        for (int c = 0; c < 6; c++) a[col][c] *= inv;
        for (int r = 0; r < 3; r++) {
            if (r == col) continue;
            cplx fct = a[r][col];
            for (int c = 0; c < 6; c++) a[r][c] -= fct * a[col][c];
        }
    }
    return a[0][3] + a[1][4] + a[2][5];
}

/* dy/dt for one beam.  sigma = +1 for the "+" branch (Eq. char_plus), -1 for "-" (Eq. char_minus):
 *   Q' = sigma c P/|P|,  P' = -sigma |P| grad c
 *   (dzQ)' = sigma [ dzQ (grad c (x) P)/|P| + c dzP (I/|P| - P (x) P/|P|^3) ]      (Eq. DzDt)
 *   (dzP)' = -sigma [ |P| dzQ Hess c + dzP (P (x) grad c)/|P| ]                     (Eq. DzDt)
 *   Z = dzQ + i dzP,  gamma = sigma grad c . P/|P| + tr(Z^{-1} Z')/2
 *   P:  a' = gamma a                                                              (Eq. amp_P)
 *   S:  a_sv' = gamma a_sv - a_sh (dN_sh/dt . N_sv),  a_sh' = gamma a_sh + a_sv (dN_sh/dt . N_sv)
 *                                                                                 (Eqs. amp_SV, amp_SH)
 *   S vector form: A' = gamma A - (A . d(P/|P|)/dt) P/|P| (the same law written without a frame). */
void orc_rhs(const orc_model *m, int mt, const orc_state *y, orc_state *f)
{
    const int cls = META_CLS(mt), wave = cls >= 2;
    const double sgm = (cls & 1) ? -1.0 : 1.0;
    double cf[10];
    orc_model_eval(m, wave, y->Q, cf);
    const double c = cf[0];
    const double g[3] = {cf[1], cf[2], cf[3]};
    const double Hs[3][3] = {{cf[4], cf[5], cf[6]}, {cf[5], cf[7], cf[8]}, {cf[6], cf[8], cf[9]}};
    const double pn = norm3(y->P);
    double Ph[3];
    for (int d = 0; d < 3; d++) Ph[d] = y->P[d] / pn;

    for (int d = 0; d < 3; d++) {
        f->Q[d] = sgm * c * Ph[d];
        f->P[d] = -sgm * pn * g[d];
    }
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) {
            cplx t1 = 0, t2 = 0, t3 = 0, t4 = 0;
            for (int l = 0; l < 3; l++) {
                double gp = g[l] * y->P[j] / pn;                                   /* (grad c (x) P)_lj / |P| */
                double proj = ((l == j) ? 1.0 / pn : 0.0) - y->P[l] * y->P[j] / (pn * pn * pn);
                t1 += y->DQ[3 * mm + l] * gp;
                t2 += y->DP[3 * mm + l] * proj;
                t3 += y->DQ[3 * mm + l] * Hs[l][j];
                t4 += y->DP[3 * mm + l] * (y->P[l] * g[j] / pn);                   /* (P (x) grad c)_lj / |P| */
            }
            f->DQ[3 * mm + j] = sgm * (t1 + c * t2);
            f->DP[3 * mm + j] = -sgm * (pn * t3 + t4);
        }
    cplx Z[9], Zd[9];
    for (int i = 0; i < 9; i++) {
        Z[i] = y->DQ[i] + I * y->DP[i];
        Zd[i] = f->DQ[i] + I * f->DP[i];
    }
    cplx gam = sgm * (g[0] * Ph[0] + g[1] * Ph[1] + g[2] * Ph[2]) + 0.5 * trace_solve(Z, Zd);
    if (!wave) {
        f->a[0] = gam * y->a[0];
        f->a[1] = 0;
        f->a[2] = 0;
    } else if (!(mt & META_VECTOR)) {
        double Nsv[3], Nsh[3], vn;
        int ref_e1 = (mt & META_REF_E1) != 0;
        s_frame(y->P, ref_e1, Nsv, Nsh, &vn);
        /* N_sh = (e x P)/|e x P|, so dN_sh/dt . N_sv = (e x P') . N_sv / |e x P| (N_sv is normal to N_sh) */
        double e[3] = {ref_e1 ? 1.0 : 0.0, 0.0, ref_e1 ? 0.0 : 1.0}, ePd[3];
        cross3(e, f->P, ePd);
        double omega = (ePd[0] * Nsv[0] + ePd[1] * Nsv[1] + ePd[2] * Nsv[2]) / vn;
        f->a[0] = gam * y->a[0] - y->a[1] * omega;
        f->a[1] = gam * y->a[1] + y->a[0] * omega;
        f->a[2] = 0;
    } else {
        double dPh[3], pdot = Ph[0] * f->P[0] + Ph[1] * f->P[1] + Ph[2] * f->P[2];
        for (int d = 0; d < 3; d++) dPh[d] = (f->P[d] - Ph[d] * pdot) / pn;
        cplx adp = y->a[0] * dPh[0] + y->a[1] * dPh[1] + y->a[2] * dPh[2];
        for (int d = 0; d < 3; d++) f->a[d] = gam * y->a[d] - adp * Ph[d];
    }
}

/* y <- y + h * d (on the 48 reals of the state) */
static void axpy_state(orc_state *out, const orc_state *y, double h, const orc_state *d)
{
    const double *yy = (const double *)y, *dd = (const double *)d;
    double *o = (double *)out;
    for (int i = 0; i < 48; i++) o[i] = yy[i] + h * dd[i];
}

/* classical RK4: y_{n+1} = y_n + dt/6 (k1 + 2 k2 + 2 k3 + k4), with k1 given (= f(y_n)) */
static void rk4_step(const orc_model *m, int mt, const orc_state *y, const orc_state *k1, double dt, orc_state *yn)
{
    orc_state k2, k3, k4, tmp;
    axpy_state(&tmp, y, 0.5 * dt, k1);
    orc_rhs(m, mt, &tmp, &k2);
    axpy_state(&tmp, y, 0.5 * dt, &k2);
    orc_rhs(m, mt, &tmp, &k3);
    axpy_state(&tmp, y, dt, &k3);
    orc_rhs(m, mt, &tmp, &k4);
    const double *yy = (const double *)y, *a1 = (const double *)k1, *a2 = (const double *)&k2,
                 *a3 = (const double *)&k3, *a4 = (const double *)&k4;
    double *o = (double *)yn;
    for (int i = 0; i < 48; i++) o[i] = yy[i] + dt / 6.0 * (a1[i] + 2.0 * a2[i] + 2.0 * a3[i] + a4[i]);
}

/* Reconstruction record of a beam at a sample time inside step [t_n, t_n + dt]:
 * Q and P by cubic Hermite interpolation from (y, y', y1, y1'), amplitudes linearly in theta;
 * then the polarised amplitude times the quadrature weight w:
 *   P: w a P/|P|;  S: w (a_sv N_sv + a_sh N_sh);  S vector form: w A.
 * rec = Q(3), P(3), A(3 complex interleaved). */
static void make_record(int mt, const orc_state *y0, const orc_state *f0, const orc_state *y1,
                        const orc_state *f1, double dt, double th, double w, double rec[12])
{
    const double h00 = 2 * th * th * th - 3 * th * th + 1, h10 = th * th * th - 2 * th * th + th;
    const double h01 = -2 * th * th * th + 3 * th * th, h11 = th * th * th - th * th;
    double Q[3], P[3];
    for (int d = 0; d < 3; d++) {
        Q[d] = h00 * y0->Q[d] + h10 * dt * f0->Q[d] + h01 * y1->Q[d] + h11 * dt * f1->Q[d];
        P[d] = h00 * y0->P[d] + h10 * dt * f0->P[d] + h01 * y1->P[d] + h11 * dt * f1->P[d];
    }
    cplx a[3];
    for (int j = 0; j < 3; j++) a[j] = (1.0 - th) * y0->a[j] + th * y1->a[j];
    cplx A[3];
    const int cls = META_CLS(mt);
    if (cls < 2) {
        double pn = norm3(P);
        for (int d = 0; d < 3; d++) A[d] = w * a[0] * (P[d] / pn);
    } else if (!(mt & META_VECTOR)) {
        double Nsv[3], Nsh[3];
        s_frame(P, (mt & META_REF_E1) != 0, Nsv, Nsh, NULL);
        for (int d = 0; d < 3; d++) A[d] = w * (a[0] * Nsv[d] + a[1] * Nsh[d]);
    } else {
        for (int d = 0; d < 3; d++) A[d] = w * a[d];
    }
    for (int d = 0; d < 3; d++) {
        rec[d] = Q[d];
        rec[3 + d] = P[d];
        rec[6 + 2 * d] = creal(A[d]);
        rec[7 + 2 * d] = cimag(A[d]);
    }
}

/* Advance nb beams nsteps RK4 steps of size dt (Sec. 2.3).  Sample j is taken inside step
 * s_step[j] at fraction s_theta[j] in [0,1] (samples sorted by step); its record goes to
 * rec[(j*nb + b)*12].  States are updated in place. */
void orc_propagate(const orc_model *m, int nb, double *st_, const int *meta, double dt, int nsteps,
                   int ns, const int *s_step, const double *s_theta, double w, double *rec)
{
    orc_state *st = (orc_state *)st_;
#pragma omp parallel for schedule(dynamic, 16)
    for (int b = 0; b < nb; b++) {
        orc_state y = st[b], f0, y1, f1;
        const int mt = meta[b];
        orc_rhs(m, mt, &y, &f0);
        int j = 0;
        for (int n = 0; n < nsteps; n++) {
            rk4_step(m, mt, &y, &f0, dt, &y1);
            orc_rhs(m, mt, &y1, &f1);
            while (j < ns && s_step[j] == n) {
                make_record(mt, &y, &f0, &y1, &f1, dt, s_theta[j], w, rec + ((size_t)j * nb + b) * 12);
                j++;
            }
            y = y1;
            f0 = f1;
        }
        st[b] = y;
    }
}

/* records of the current states (theta = 0 of a zero-length step) */
void orc_records(int nb, const double *st_, const int *meta, double w, double *rec)
{
    const orc_state *st = (const orc_state *)st_;
    for (int b = 0; b < nb; b++) make_record(meta[b], st + b, st + b, st + b, st + b, 0.0, 0.0, w, rec + (size_t)b * 12);
}

void orc_rhs_many(const orc_model *m, int nb, const double *st_, const int *meta, double *out_)
{
    const orc_state *st = (const orc_state *)st_;
    orc_state *out = (orc_state *)out_;
    for (int b = 0; b < nb; b++) orc_rhs(m, meta[b], st + b, out + b);
}

/* ------------------------------------------------------------------------- */
/* Gaussian summation, Eq. FGA                                                */
/* ------------------------------------------------------------------------- */
/* u(x) = sum_b A_b exp(i k P_b.(x-Q_b) - k|x-Q_b|^2/2), over every beam (rw <= 0) or only the
 * beams with |x - Q_b| <= rw.  u is complex [nx][3]. */
void orc_gauss_sum(int nb, const double *rec, double k, double rw, int nx, const double *x, double *u_)
{
    cplx *u = (cplx *)u_;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < nx; i++) {
        cplx acc[3] = {0, 0, 0};
        const double *xi = x + 3 * i;
        for (int b = 0; b < nb; b++) {
            const double *r = rec + (size_t)b * 12;
            double dx[3] = {xi[0] - r[0], xi[1] - r[1], xi[2] - r[2]};
            double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
            if (rw > 0.0 && r2 > rw * rw) continue;
            double ph = r[3] * dx[0] + r[4] * dx[1] + r[5] * dx[2];
            cplx e = cexp(I * k * ph - 0.5 * k * r2);
            for (int d = 0; d < 3; d++) acc[d] += (r[6 + 2 * d] + I * r[7 + 2 * d]) * e;
        }
        for (int d = 0; d < 3; d++) u[(size_t)i * 3 + d] = acc[d];
    }
}

/* ------------------------------------------------------------------------- */
/* cell binning                                                               */
/* ------------------------------------------------------------------------- */
/* key = cell id of an FP32 centre: cell_d = floor((Q_d - o_d) * inv_h) evaluated in FP32
 * round-to-nearest (one subtraction, one multiplication, no fused multiply-add),
 * clamped to [0, nc_d - 1]; id = (c0 nc1 + c1) nc2 + c2.  Q is float [nb][3]. */
void orc_bin_keys_f32(int nb, const float *Q, const float o[3], float inv_h, const int nc[3], int32_t *key)
{
    for (int b = 0; b < nb; b++) {
        int cell[3];
        for (int d = 0; d < 3; d++) {
            volatile float diff = Q[3 * b + d] - o[d];
            volatile float t = diff * inv_h;
            float fl = floorf(t);
            int cd;
            if (!(fl >= 0.0f)) cd = 0;              /* negative or NaN */
            else if (fl > (float)(nc[d] - 1)) cd = nc[d] - 1;
            else cd = (int)fl;
            cell[d] = cd;
        }
        key[b] = (cell[0] * nc[1] + cell[1]) * nc[2] + cell[2];
    }
}

/* stable counting sort of beam ids by key: perm lists beams cell by cell, in increasing id
 * inside a cell; cell_start has ncells + 1 entries. */
void orc_bin_sort(int nb, const int32_t *key, int ncells, int32_t *perm, int32_t *cell_start)
{
    int32_t *cnt = (int32_t *)calloc((size_t)ncells + 1, sizeof(int32_t));
    for (int b = 0; b < nb; b++) cnt[key[b] + 1]++;
    for (int c = 0; c < ncells; c++) cnt[c + 1] += cnt[c];
    memcpy(cell_start, cnt, sizeof(int32_t) * ((size_t)ncells + 1));
    for (int b = 0; b < nb; b++) perm[cnt[key[b]]++] = b;
    free(cnt);
}
