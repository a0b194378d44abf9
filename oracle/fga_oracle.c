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
 *   - flat-interface events: Snell's law, the printed Zoeppritz (Sec. 3.1, Eqs. p:int, Yilmaz, Inter_DzQDzP)
 *     system in angle variables, the F-W jump of dzQ and dzP
 *
 * Readings of points the paper leaves open:
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
    int shells;             /* layered medium with spherical interfaces |x - ctr| = zif[i] (radii, decreasing) */
    double ctr[3];
    int undul;              /* layered medium with undulating interfaces x3 = zif[i] + uamp[i] cos(uk0 x1) cos(uk1 x2) */
    double uk[2];
    const double *uamp;
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

/* Layer of a point: flat layers by depth x3 (a point on an interface belongs to the deeper layer);
 * spherical layers by the number of spheres that enclose the point (a point on a sphere is inside it);
 * undulating layers by the number of surfaces at or above the point. */
static int layer_of(const orc_model *m, const double x[3])
{
    int l = 0;
    if (m->shells) {
        const double r = sqrt((x[0] - m->ctr[0]) * (x[0] - m->ctr[0]) + (x[1] - m->ctr[1]) * (x[1] - m->ctr[1]) +
                              (x[2] - m->ctr[2]) * (x[2] - m->ctr[2]));
        while (l < m->nlay - 1 && r <= m->zif[l]) l++;
        return l;
    }
    if (m->undul) {
        const double cc = cos(m->uk[0] * x[0]) * cos(m->uk[1] * x[1]);
        while (l < m->nlay - 1 && x[2] >= m->zif[l] + m->uamp[l] * cc) l++;
        return l;
    }
    while (l < m->nlay - 1 && x[2] >= m->zif[l]) l++;
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
        int l = layer_of(m, x);
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
 * bit 3: S amplitude carried as a complex 3-vector (parallel-transport form),
 * bits 4-7: layer of the beam (layered media), bits 8-11: interfaces crossed so far */
#define META_CLS(mt) ((mt) & 3)
#define META_REF_E1 4
#define META_VECTOR 8
#define META_LAYER(mt) (((mt) >> 4) & 15)
#define META_GEN(mt) (((mt) >> 8) & 15)
#define META_ROOT(mt) (((mt) >> 13) & 3)

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
        /* layered media: layer (bits 4-7) and the class of the root beam of the lineage (bits 13-14) */
        int lay_bits = m->kind == ORC_LAYERED ? ((layer_of(m, y->Q) << 4) | (cls << 13)) : 0;
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
        meta[mi] = mt | lay_bits;
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
    if (m->kind == ORC_LAYERED) {
        /* the beam's own layer (a beam sitting on an interface belongs to the side it travels in) */
        for (int f = 0; f < 10; f++) cf[f] = 0.0;
        cf[0] = wave ? m->lcs[META_LAYER(mt)] : m->lcp[META_LAYER(mt)];
    } else {
        orc_model_eval(m, wave, y->Q, cf);
    }
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

/* ------------------------------------------------------------------------- */
/* flat interfaces (Sec. 3.1)                                                 */
/* ------------------------------------------------------------------------- */
/* A beam crossing the plane x3 = zif from layer 1 (the incident side) into layer 2 scatters into up
 * to four beams: reflected P and S (back into layer 1) and transmitted P and S (into layer 2).
 *
 * Snell's law, Eq. p:int: every child keeps the horizontal part of P and the frequency c|P| of the
 * incident beam, and its vertical component is p_z' = +-sqrt((p_z n)^2 + (n^2 - 1)(p_x^2 + p_y^2))
 * with n = c_in / c_child (n_1, n_2, n_3 of the paper for a P incidence); reflected children flip the
 * sign of p_z, transmitted ones keep it.
 *
 * Amplitudes: the Zoeppritz system as printed, Eq. Yilmaz.  It is written in the plane of incidence
 * of a P wave, with the P angles theta and the S angles phi measured from the interface normal, for
 * potential amplitudes (a wave of speed c and potential amplitude X has displacement amplitude
 * proportional to X / c; every matrix entry carries that scaling).  Readings:
 *   - the last entry of the printed right-hand side, cos(2 theta_r), is garbled: the shear-traction
 *     row of the same matrix needs sin(2 theta_r), and only sin gives no converted S wave at normal
 *     incidence;
 *   - SV incidence (the paper: "handled similarly"): the same matrix, whose columns are the four
 *     outgoing waves, with the incident S wave's column as right-hand side,
 *     (-(a1/b1) sin phi, (a1/b1) cos phi, -sin 2phi, (a1/b1)^2 cos 2phi), phi its angle;
 *   - SH incidence (no P-S interaction, as the paper notes): the textbook coefficients of a welded
 *     interface for displacement, R = (r1 b1 cos phi1 - r2 b2 cos phi2) / D, T = 2 r1 b1 cos phi1 / D,
 *     D = r1 b1 cos phi1 + r2 b2 cos phi2;
 *   - a beam in 3-D: the plane of incidence is spanned by the horizontal direction h of the beam's
 *     direction of travel V = sigma P (sigma = -1 on the "-" branch, whose beams move along -P) and by
 *     the normal nrm = sign(V_3) e3 pointing into layer 2.  A wave travelling along d = d_h h + d_n nrm
 *     is polarised along d (P), along d_n h - d_h nrm (SV, the sign convention of the printed
 *     matrix) or along s = nrm x h (SH);
 *   - beyond a critical angle the cosine of that wave's angle is i sigma sqrt(sin^2 - 1), so that it
 *     decays away from the interface; it takes part in the system but is not created as a beam.
 *
 * dzQ and dzP jump by Eq. Inter_DzQDzP: dzQ' = dzQ F, dzP' = dzP W with W = F^{-T}; its grad c term
 * vanishes between homogeneous layers. */

/* 4x4 complex solve by Gaussian elimination with partial pivoting; returns 0 if singular */
static int solve4(cplx A[4][4], cplx b[4], cplx x[4])
{
    for (int c = 0; c < 4; c++) {
        int piv = c;
        for (int r = c + 1; r < 4; r++)
            if (cabs(A[r][c]) > cabs(A[piv][c])) piv = r;
        if (cabs(A[piv][c]) < 1e-300) return 0;
        for (int j = 0; j < 4; j++) {
            cplx t = A[c][j];
            A[c][j] = A[piv][j];
            A[piv][j] = t;
        }
        cplx t = b[c];
        b[c] = b[piv];
        b[piv] = t;
        for (int r = c + 1; r < 4; r++) {
            cplx f = A[r][c] / A[c][c];
            for (int j = c; j < 4; j++) A[r][j] -= f * A[c][j];
            b[r] -= f * b[c];
        }
    }
    for (int r = 3; r >= 0; r--) {
        cplx s = b[r];
        for (int j = r + 1; j < 4; j++) s -= A[r][j] * x[j];
        x[r] = s / A[r][r];
    }
    return 1;
}

/* Children of beam y (meta mt, in layer la) that reached the interface to layer lb; at most 4,
 * written in the order reflected P, reflected S, transmitted P, transmitted S (propagating ones
 * whose displacement amplitude is at least rel_min of the incident one).  Returns the count. */
int orc_interface_event(const orc_model *m, int mt, const double *y_, int lb, double rel_min, double *out_, int *meta_out)
{
    const orc_state *y = (const orc_state *)y_;
    orc_state *out = (orc_state *)out_;
    const int la = META_LAYER(mt), cls = META_CLS(mt), swave = cls >= 2;
    const double sigma = (cls & 1) ? -1.0 : 1.0;
    /* layer 1 is the incident side (the paper's "^" side for its downgoing P wave), layer 2 the other */
    const double a1 = m->lcp[la], b1 = m->lcs[la], r1 = m->lrho[la];
    const double a2 = m->lcp[lb], b2 = m->lcs[lb], r2 = m->lrho[lb];
    const double cin = swave ? b1 : a1;
    const double px = y->P[0], py = y->P[1], pz = y->P[2];
    const double pin = norm3(y->P), om = cin * pin, ph = sqrt(px * px + py * py);

    /* incident displacement vector */
    cplx U[3];
    if (!swave) {
        for (int d = 0; d < 3; d++) U[d] = y->a[0] * (y->P[d] / pin);
    } else if (mt & META_VECTOR) {
        for (int d = 0; d < 3; d++) U[d] = y->a[d];
    } else {
        double Nsv[3], Nsh[3];
        s_frame(y->P, (mt & META_REF_E1) != 0, Nsv, Nsh, NULL);
        for (int d = 0; d < 3; d++) U[d] = y->a[0] * Nsv[d] + y->a[1] * Nsh[d];
    }

    /* plane of incidence of the direction of travel */
    double h[3] = {1.0, 0.0, 0.0}, nrm[3] = {0.0, 0.0, sigma * pz >= 0.0 ? 1.0 : -1.0}, s[3];
    if (ph > 0.0) {
        h[0] = sigma * px / ph;
        h[1] = sigma * py / ph;
    }
    cross3(nrm, h, s);

    /* the outgoing waves w = 0 rP, 1 rS, 2 tP, 3 tS: Snell's law and the angles from the normal */
    const double cw[4] = {a1, b1, a2, b2};
    double pzw[4], sn[4];
    cplx cs[4];
    int prop[4];
    for (int w = 0; w < 4; w++) {
        const double n = cin / cw[w];
        const double q = (pz * n) * (pz * n) + (n * n - 1.0) * ph * ph;
        const double side = w >= 2 ? (pz >= 0.0 ? 1.0 : -1.0) : (pz >= 0.0 ? -1.0 : 1.0);
        prop[w] = q >= 0.0;
        pzw[w] = prop[w] ? side * sqrt(q) : 0.0;
        sn[w] = ph * cw[w] / om;
        const double c2 = 1.0 - sn[w] * sn[w];
        cs[w] = c2 >= 0.0 ? (cplx)sqrt(c2) : I * sigma * sqrt(-c2);
    }
    /* theta_r, phi_r, theta_t, phi_t of the printed matrix */
    const double sth_r = sn[0], sph_r = sn[1], sth_t = sn[2], sph_t = sn[3];
    const cplx cth_r = cs[0], cph_r = cs[1], cth_t = cs[2], cph_t = cs[3];
    const cplx s2th_r = 2.0 * sth_r * cth_r, s2ph_r = 2.0 * sph_r * cph_r;
    const cplx s2th_t = 2.0 * sth_t * cth_t, s2ph_t = 2.0 * sph_t * cph_t;
    const double c2ph_r = 1.0 - 2.0 * sph_r * sph_r, c2ph_t = 1.0 - 2.0 * sph_t * sph_t;
    cplx M[4][4] = {
        {cth_r, a1 / b1 * sph_r, a1 / a2 * cth_t, -a1 / b2 * sph_t},
        {-sth_r, a1 / b1 * cph_r, a1 / a2 * sth_t, a1 / b2 * cph_t},
        {-c2ph_r, -s2ph_r, r2 / r1 * c2ph_t, -r2 / r1 * s2ph_t},
        {s2th_r, -(a1 / b1) * (a1 / b1) * c2ph_r, r2 * a1 * a1 * b2 * b2 / (r1 * a2 * a2 * b1 * b1) * s2th_t,
         r2 * a1 * a1 / (r1 * b1 * b1) * c2ph_t}};
    /* incident amplitude along its own polarisation in the plane of incidence */
    const double din_h = ph / pin, din_n = fabs(pz) / pin;       /* V/|V| = din_h h + din_n nrm */
    cplx rhs[4], X[4];
    cplx Csh = 0.0;
    if (!swave) {
        cplx A = 0.0;
        for (int d = 0; d < 3; d++) A += U[d] * (din_h * h[d] + din_n * nrm[d]);
        rhs[0] = cth_r * A;
        rhs[1] = sth_r * A;
        rhs[2] = c2ph_r * A;
        rhs[3] = s2th_r * A;
    } else {
        cplx B = 0.0;
        for (int d = 0; d < 3; d++) {
            B += U[d] * (din_n * h[d] - din_h * nrm[d]);
            Csh += U[d] * s[d];
        }
        rhs[0] = -a1 / b1 * sph_r * B;
        rhs[1] = a1 / b1 * cph_r * B;
        rhs[2] = -s2ph_r * B;
        rhs[3] = (a1 / b1) * (a1 / b1) * c2ph_r * B;
    }
    if (!solve4(M, rhs, X)) return 0;
    /* SH: reflected and transmitted displacement factors (zero for a P incidence) */
    const cplx Dsh = r1 * b1 * cph_r + r2 * b2 * cph_t;
    const cplx Rsh = (r1 * b1 * cph_r - r2 * b2 * cph_t) / Dsh, Tsh = 2.0 * r1 * b1 * cph_r / Dsh;

    double ain = 0.0;
    for (int d = 0; d < 3; d++) ain += creal(U[d] * conj(U[d]));
    ain = sqrt(ain);
    int nout = 0;
    for (int w = 0; w < 4; w++) {
        if (!prop[w]) continue;
        const int s_wave = w & 1, trans = w >= 2;
        /* direction of travel of the child in the plane of incidence, and its displacement vector */
        const double dh = sn[w], dn = trans ? creal(cs[w]) : -creal(cs[w]);
        const double amp = cin / cw[w];                /* potential -> displacement amplitude */
        cplx Uc[3];
        for (int d = 0; d < 3; d++) {
            if (!s_wave) {
                Uc[d] = amp * X[w] * (dh * h[d] + dn * nrm[d]);
            } else {
                Uc[d] = amp * X[w] * (dn * h[d] - dh * nrm[d]);
                if (swave) Uc[d] += (trans ? Tsh : Rsh) * Csh * s[d];
            }
        }
        double amag = 0.0;
        for (int d = 0; d < 3; d++) amag += creal(Uc[d] * conj(Uc[d]));
        amag = sqrt(amag);
        if (!(amag >= rel_min * ain) || amag == 0.0) continue;
        orc_state *c = out + nout;
        *c = *y;
        const double Pr[3] = {px, py, pzw[w]};
        for (int d = 0; d < 3; d++) c->P[d] = Pr[d];
        /* F = I except its last row ((kappa-1) p_x/p_z, (kappa-1) p_y/p_z, kappa p_z'/p_z),
         * kappa = (c_child/c_in)^2; W = F^{-T} */
        const double kap = (cw[w] / cin) * (cw[w] / cin);
        const double Fm[3][3] = {{1, 0, 0}, {0, 1, 0}, {(kap - 1.0) * px / pz, (kap - 1.0) * py / pz, kap * Pr[2] / pz}};
        const double Fi[3][3] = {{1, 0, 0}, {0, 1, 0}, {-Fm[2][0] / Fm[2][2], -Fm[2][1] / Fm[2][2], 1.0 / Fm[2][2]}};
        for (int mm = 0; mm < 3; mm++)
            for (int j = 0; j < 3; j++) {
                cplx sq = 0, sp = 0;
                for (int l = 0; l < 3; l++) {
                    sq += y->DQ[3 * mm + l] * Fm[l][j];
                    sp += y->DP[3 * mm + l] * Fi[j][l];   /* (F^{-1})^T */
                }
                c->DQ[3 * mm + j] = sq;
                c->DP[3 * mm + j] = sp;
            }
        const int cc = (s_wave ? 2 : 0) | (cls & 1);
        int mt_c = cc | ((trans ? lb : la) << 4) | ((META_GEN(mt) + 1) << 8) | (mt & (3 << 13));
        c->a[0] = c->a[1] = c->a[2] = 0;
        const double pn = norm3(Pr);
        if (!s_wave) {
            for (int d = 0; d < 3; d++) c->a[0] += Uc[d] * (Pr[d] / pn);
        } else if (mt & META_VECTOR) {
            mt_c |= META_VECTOR;
            for (int d = 0; d < 3; d++) c->a[d] = Uc[d];
        } else {
            const int r = orc_s_ref_e1(Pr);
            if (r) mt_c |= META_REF_E1;
            double fsv[3], fsh[3];
            s_frame(Pr, r, fsv, fsh, NULL);
            for (int d = 0; d < 3; d++) {
                c->a[0] += Uc[d] * fsv[d];
                c->a[1] += Uc[d] * fsh[d];
            }
        }
        meta_out[nout] = mt_c;
        nout++;
    }
    return nout;
}

/* One RK4 step of size dt for every beam of a layered medium, with interface events (Sec. 3.1):
 * a beam whose step crosses an interface is advanced to the crossing (its motion is straight in a
 * homogeneous layer), replaced by its children, and every child is advanced through the rest of the
 * step.  Beams that have crossed gmax interfaces are dropped at their next one.  The new population
 * (parents without events in input order, children in place of their parent) goes to out/meta_out,
 * with path[] recording the lineage (parent path * 4 + child slot + 1).  Returns the new count or
 * -1 if cap is too small. */
int orc_layered_step(const orc_model *m, int nb, const double *st_, const int *meta, const long long *path,
                     double dt, int gmax, double rel_min, int cap, double *out_, int *meta_out, long long *path_out,
                     int *parent_out)
{
    const orc_state *st = (const orc_state *)st_;
    orc_state *out = (orc_state *)out_;
    int n = 0;
    if (m->shells || m->undul) return -1;   /* flat layers only; curved ones step in fga_oracle.py */
    for (int b = 0; b < nb; b++) {
        const int mt = meta[b], L = META_LAYER(mt);
        orc_state y = st[b], f0, y1;
        orc_rhs(m, mt, &y, &f0);
        rk4_step(m, mt, &y, &f0, dt, &y1);
        double ztop = L > 0 ? m->zif[L - 1] : -INFINITY, zbot = L < m->nlay - 1 ? m->zif[L] : INFINITY;
        if (y1.Q[2] >= ztop && y1.Q[2] < zbot) {
            if (n >= cap) return -1;
            out[n] = y1;
            meta_out[n] = mt;
            path_out[n] = path[b];
            if (parent_out) parent_out[n] = b;
            n++;
            continue;
        }
        int down = y1.Q[2] >= zbot;
        double zc = down ? zbot : ztop;
        int lb = down ? L + 1 : L - 1;
        double th = (zc - y.Q[2]) / (y1.Q[2] - y.Q[2]);
        if (META_GEN(mt) >= gmax) continue;
        orc_state yc;
        rk4_step(m, mt, &y, &f0, th * dt, &yc);
        yc.Q[2] = zc;
        orc_state ch[4];
        int cm[4];
        int nc = orc_interface_event(m, mt, (const double *)&yc, lb, rel_min, (double *)ch, cm);
        for (int c = 0; c < nc; c++) {
            orc_state fc, ye;
            orc_rhs(m, cm[c], &ch[c], &fc);
            rk4_step(m, cm[c], &ch[c], &fc, (1.0 - th) * dt, &ye);
            if (n >= cap) return -1;
            out[n] = ye;
            meta_out[n] = cm[c];
            /* child slot: 0 rP, 1 rS, 2 tP, 3 tS */
            int slot = ((cm[c] >> 4) & 15) == L ? ((cm[c] & 2) ? 1 : 0) : ((cm[c] & 2) ? 3 : 2);
            path_out[n] = path[b] * 4 + slot + 1;
            if (parent_out) parent_out[n] = b;
            n++;
        }
    }
    return n;
}

/* One classical RK4 step of size dt for each of n beams (layered media: each in its own layer). */
void orc_rk4_many(const orc_model *m, int n, const double *st_, const int *meta, double dt, double *out_)
{
    const orc_state *st = (const orc_state *)st_;
    orc_state *out = (orc_state *)out_;
    for (int b = 0; b < n; b++) {
        orc_state f0;
        orc_rhs(m, meta[b], &st[b], &f0);
        rk4_step(m, meta[b], &st[b], &f0, dt, &out[b]);
    }
}

/* ------------------------------------------------------------------------- */
/* discrete adjoint (no counterpart in the paper, which defers its kernels to other works)  */
/* ------------------------------------------------------------------------- */
/* Reverse mode of the forward solve above for grid media, for the waveform misfit
 * L = 1/2 sum |u - d|^2 over receivers and samples, with respect to the 10 node fields of the P and
 * S grids.  Complex adjoints follow z_bar = dL/dRe z + i dL/dIm z: for w = f(z) holomorphic
 * z_bar += conj(f'(z)) w_bar, and a real r feeding w gets r_bar += Re(conj(dw/dr) w_bar). */

/* trilinear weights of a grid point and their derivatives along each axis (zero where clamped) */
static void grid_weights(const orc_model *m, const double x[3], size_t node[8], double wgt[8], double dw[8][3])
{
    int i[3];
    double fr[3], dfr[3];
    for (int d = 0; d < 3; d++) {
        double t = (x[d] - m->o[d]) / m->h[d];
        dfr[d] = 1.0 / m->h[d];
        if (t < 0.0) {
            t = 0.0;
            dfr[d] = 0.0;
        }
        if (t > (double)(m->n[d] - 1)) {
            t = (double)(m->n[d] - 1);
            dfr[d] = 0.0;
        }
        int id = (int)floor(t);
        if (id > m->n[d] - 2) id = m->n[d] - 2;
        i[d] = id;
        fr[d] = t - (double)id;
    }
    int c = 0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int e = 0; e < 2; e++, c++) {
                double w0 = a ? fr[0] : 1.0 - fr[0], w1 = b ? fr[1] : 1.0 - fr[1], w2 = e ? fr[2] : 1.0 - fr[2];
                double s0 = a ? 1.0 : -1.0, s1 = b ? 1.0 : -1.0, s2 = e ? 1.0 : -1.0;
                node[c] = ((size_t)(i[0] + a) * m->n[1] + (size_t)(i[1] + b)) * m->n[2] + (size_t)(i[2] + e);
                wgt[c] = w0 * w1 * w2;
                dw[c][0] = s0 * dfr[0] * w1 * w2;
                dw[c][1] = w0 * s1 * dfr[1] * w2;
                dw[c][2] = w0 * w1 * s2 * dfr[2];
            }
}

/* adjoint of the model fields at Q: Q_bar += sum_f cbar[f] d field_f/dQ; node grads += weights cbar */
static void model_vjp(const orc_model *m, int wave, const double Q[3], const double cbar[10], double Qbar[3],
                      double *gp, double *gs)
{
    if (m->kind != ORC_GRID) return; /* constant media: the fields do not depend on Q or on nodes */
    size_t node[8];
    double wgt[8], dw[8][3];
    grid_weights(m, Q, node, wgt, dw);
    const float *g = wave ? m->gs : m->gp;
    double *G = wave ? gs : gp;
    for (int c = 0; c < 8; c++)
        for (int f = 0; f < 10; f++) {
            const double v = (double)g[node[c] * 10 + f];
            for (int d = 0; d < 3; d++) Qbar[d] += cbar[f] * v * dw[c][d];
            if (G) {
                const double add = cbar[f] * wgt[c];
#pragma omp atomic
                G[node[c] * 10 + f] += add;
            }
        }
}

/* ybar += (d rhs/dy)^T fbar; model adjoints scattered onto the node grids gp/gs (may be NULL) */
void orc_rhs_vjp(const orc_model *m, int mt, const orc_state *y, const orc_state *fb, orc_state *yb, double *gp,
                 double *gs)
{
    const int cls = META_CLS(mt), wave = cls >= 2;
    const double sg = (cls & 1) ? -1.0 : 1.0;
    double cf[10];
    orc_model_eval(m, wave, y->Q, cf);
    const double c = cf[0];
    const double g[3] = {cf[1], cf[2], cf[3]};
    const double H[3][3] = {{cf[4], cf[5], cf[6]}, {cf[5], cf[7], cf[8]}, {cf[6], cf[8], cf[9]}};
    const double pn = norm3(y->P), ip = 1.0 / pn;
    double Ph[3];
    for (int d = 0; d < 3; d++) Ph[d] = y->P[d] * ip;
    const double cip = c * ip;
    /* forward intermediates */
    cplx u[3], v[3], t3[3][3], fDQ[3][3], fDP[3][3];
    for (int mm = 0; mm < 3; mm++) {
        u[mm] = 0;
        v[mm] = 0;
        for (int l = 0; l < 3; l++) {
            u[mm] += y->DQ[3 * mm + l] * g[l];
            v[mm] += y->DP[3 * mm + l] * Ph[l];
        }
        for (int j = 0; j < 3; j++) {
            t3[mm][j] = 0;
            for (int l = 0; l < 3; l++) t3[mm][j] += y->DQ[3 * mm + l] * H[l][j];
            fDQ[mm][j] = sg * (u[mm] * Ph[j] + cip * y->DP[3 * mm + j] - cip * v[mm] * Ph[j]);
            fDP[mm][j] = -sg * (pn * t3[mm][j] + v[mm] * g[j]);
        }
    }
    double fP[3];
    for (int d = 0; d < 3; d++) fP[d] = -sg * pn * g[d];
    cplx Z[9], Zd[9], Zi[9];
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) {
            Z[3 * mm + j] = y->DQ[3 * mm + j] + I * y->DP[3 * mm + j];
            Zd[3 * mm + j] = fDQ[mm][j] + I * fDP[mm][j];
        }
    /* Z^{-1} by Gauss-Jordan on [Z | I] */
    {
        cplx a[3][6];
        for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++) {
                a[r][q] = Z[3 * r + q];
                a[r][3 + q] = (r == q) ? 1.0 : 0.0;
            }
        for (int col = 0; col < 3; col++) {
            int piv = col;
            for (int r = col + 1; r < 3; r++)
                if (cabs(a[r][col]) > cabs(a[piv][col])) piv = r;
            for (int q = 0; q < 6; q++) {
                cplx t = a[col][q];
                a[col][q] = a[piv][q];
                a[piv][q] = t;
            }
            cplx inv = 1.0 / a[col][col];
            for (int q = 0; q < 6; q++) a[col][q] *= inv;
            for (int r = 0; r < 3; r++) {
                if (r == col) continue;
                cplx fct = a[r][col];
                for (int q = 0; q < 6; q++) a[r][q] -= fct * a[col][q];
            }
        }
        for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++) Zi[3 * r + q] = a[r][3 + q];
    }
    cplx tr = 0;
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) tr += Zi[3 * j + mm] * Zd[3 * mm + j];
    const cplx gam = sg * (g[0] * Ph[0] + g[1] * Ph[1] + g[2] * Ph[2]) + 0.5 * tr;

    /* adjoint accumulators */
    double cb[10] = {0}, Phb[3] = {0}, pnb = 0, cipb = 0, fPb[3];
    cplx fDQb[3][3], fDPb[3][3], ub[3] = {0}, vb[3] = {0}, t3b[3][3];
    for (int d = 0; d < 3; d++) fPb[d] = fb->P[d];
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) {
            fDQb[mm][j] = fb->DQ[3 * mm + j];
            fDPb[mm][j] = fb->DP[3 * mm + j];
        }
    /* amplitudes */
    cplx gamb = 0;
    if (!wave) {
        yb->a[0] += conj(gam) * fb->a[0];
        gamb = conj(y->a[0]) * fb->a[0];
    } else {
        /* omega = -s1 s2 / D, s1 = fP.(e x P), s2 = e.P, D = |P|^3 - s2^2 |P| */
        const int r1 = (mt & META_REF_E1) != 0;
        const double e[3] = {r1 ? 1.0 : 0.0, 0.0, r1 ? 0.0 : 1.0};
        double exP[3], fPxe[3];
        cross3(e, y->P, exP);
        cross3(fP, e, fPxe);
        const double s1 = fP[0] * exP[0] + fP[1] * exP[1] + fP[2] * exP[2];
        const double s2 = e[0] * y->P[0] + e[1] * y->P[1] + e[2] * y->P[2];
        const double D = pn * pn * pn - s2 * s2 * pn;
        const double om = -s1 * s2 / D;
        yb->a[0] += conj(gam) * fb->a[0] + om * fb->a[1];
        yb->a[1] += conj(gam) * fb->a[1] - om * fb->a[0];
        gamb = conj(y->a[0]) * fb->a[0] + conj(y->a[1]) * fb->a[1];
        const double omb = creal(-conj(y->a[1]) * fb->a[0] + conj(y->a[0]) * fb->a[1]);
        /* d omega / d fP = -(s2/D) e x P;  d omega / dP = -(s2/D) fP x e - (s1/D) e + (s1 s2/D^2) dD/dP */
        for (int d = 0; d < 3; d++) {
            fPb[d] += omb * (-(s2 / D) * exP[d]);
            const double dD = 3.0 * pn * y->P[d] - 2.0 * s2 * pn * e[d] - s2 * s2 * y->P[d] / pn;
            yb->P[d] += omb * (-(s2 / D) * fPxe[d] - (s1 / D) * e[d] + (s1 * s2 / (D * D)) * dD);
        }
    }
    /* gamma = sg g.Ph + tr/2 */
    for (int d = 0; d < 3; d++) {
        cb[1 + d] += sg * Ph[d] * creal(gamb);
        Phb[d] += sg * g[d] * creal(gamb);
    }
    const cplx trb = 0.5 * gamb;
    /* tr = sum_mj Zi_jm Zd_mj: Zd_bar = conj(Zi^T) trb, Z_bar = -conj((Zi Zd Zi)^T) trb */
    cplx ZiZdZi[9];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) {
            cplx s = 0;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) s += Zi[3 * r + a] * Zd[3 * a + b] * Zi[3 * b + q];
            ZiZdZi[3 * r + q] = s;
        }
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) {
            const cplx zdb = conj(Zi[3 * j + mm]) * trb;
            const cplx zb = -conj(ZiZdZi[3 * j + mm]) * trb;
            fDQb[mm][j] += zdb;
            fDPb[mm][j] += -I * zdb;
            yb->DQ[3 * mm + j] += zb;
            yb->DP[3 * mm + j] += -I * zb;
        }
    /* fDP = -sg (pn t3 + v g) */
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) {
            pnb += creal(conj(-sg * t3[mm][j]) * fDPb[mm][j]);
            t3b[mm][j] = -sg * pn * fDPb[mm][j];
            vb[mm] += -sg * g[j] * fDPb[mm][j];
            cb[1 + j] += creal(conj(-sg * v[mm]) * fDPb[mm][j]);
        }
    /* t3 = DQ H */
    for (int mm = 0; mm < 3; mm++)
        for (int l = 0; l < 3; l++)
            for (int j = 0; j < 3; j++) {
                yb->DQ[3 * mm + l] += H[l][j] * t3b[mm][j];
                const double hb = creal(conj(y->DQ[3 * mm + l]) * t3b[mm][j]);
                /* H_lj is field 4.. (symmetric storage) */
                static const int hidx[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
                cb[hidx[l][j]] += hb;
            }
    /* fDQ = sg (u Ph + cip DP - cip v Ph) */
    for (int mm = 0; mm < 3; mm++)
        for (int j = 0; j < 3; j++) {
            const cplx b = fDQb[mm][j];
            ub[mm] += sg * Ph[j] * b;
            yb->DP[3 * mm + j] += sg * cip * b;
            vb[mm] += -sg * cip * Ph[j] * b;
            cipb += creal(conj(sg * (y->DP[3 * mm + j] - v[mm] * Ph[j])) * b);
            Phb[j] += creal(conj(sg * (u[mm] - cip * v[mm])) * b);
        }
    /* u = DQ g, v = DP Ph */
    for (int mm = 0; mm < 3; mm++)
        for (int l = 0; l < 3; l++) {
            yb->DQ[3 * mm + l] += g[l] * ub[mm];
            cb[1 + l] += creal(conj(y->DQ[3 * mm + l]) * ub[mm]);
            yb->DP[3 * mm + l] += Ph[l] * vb[mm];
            Phb[l] += creal(conj(y->DP[3 * mm + l]) * vb[mm]);
        }
    /* fP = -sg pn g, fQ = sg c Ph */
    for (int d = 0; d < 3; d++) {
        pnb += -sg * g[d] * fPb[d];
        cb[1 + d] += -sg * pn * fPb[d];
        cb[0] += sg * Ph[d] * fb->Q[d];
        Phb[d] += sg * c * fb->Q[d];
    }
    /* cip = c / pn */
    cb[0] += ip * cipb;
    pnb += -c * ip * ip * cipb;
    /* Ph = P / pn, pn = |P| */
    double phd = Phb[0] * Ph[0] + Phb[1] * Ph[1] + Phb[2] * Ph[2];
    for (int d = 0; d < 3; d++) yb->P[d] += (Phb[d] - Ph[d] * phd) * ip + pnb * Ph[d];
    model_vjp(m, wave, y->Q, cb, yb->Q, gp, gs);
}

/* adjoint of the S frame: given Nsv_bar, Nsh_bar, add the cotangent of P (Nsh = e x P/|e x P|, Nsv = Nsh x P^) */
static void s_frame_vjp(const double P[3], int ref_e1, const double Nsvb[3], const double Nshb[3], double Pb[3])
{
    const double e[3] = {ref_e1 ? 1.0 : 0.0, 0.0, ref_e1 ? 0.0 : 1.0};
    double v[3], Nsh[3], Ph[3], Nshb2[3], Phb[3], vb[3], tmp[3];
    cross3(e, P, v);
    const double nv = norm3(v), nP = norm3(P);
    for (int d = 0; d < 3; d++) {
        Nsh[d] = v[d] / nv;
        Ph[d] = P[d] / nP;
    }
    /* Nsv = Nsh x Ph: Nsh_bar += Ph x Nsv_bar, Ph_bar = Nsv_bar x Nsh */
    cross3(Ph, Nsvb, tmp);
    for (int d = 0; d < 3; d++) Nshb2[d] = Nshb[d] + tmp[d];
    cross3(Nsvb, Nsh, Phb);
    const double s1 = Nsh[0] * Nshb2[0] + Nsh[1] * Nshb2[1] + Nsh[2] * Nshb2[2];
    for (int d = 0; d < 3; d++) vb[d] = (Nshb2[d] - Nsh[d] * s1) / nv;
    /* v = e x P: P_bar += v_bar x e */
    cross3(vb, e, tmp);
    const double s2 = Ph[0] * Phb[0] + Ph[1] * Phb[1] + Ph[2] * Phb[2];
    for (int d = 0; d < 3; d++) Pb[d] += tmp[d] + (Phb[d] - Ph[d] * s2) / nP;
}

/* cotangent of one record from the receiver cotangents ub [nx][3] (complex) of its sample:
 * u(x) = sum A exp(phi), phi = i k P.(x-Q) - k|x-Q|^2/2 inside the window |x-Q| <= rw (rw <= 0: no window). */
static void gauss_vjp_record(const double r[12], double k, double rw, int nx, const double *x, const cplx *ub,
                             double rb[12])
{
    cplx Ab[3] = {0, 0, 0};
    double Qb[3] = {0, 0, 0}, Pb[3] = {0, 0, 0};
    const cplx A[3] = {r[6] + I * r[7], r[8] + I * r[9], r[10] + I * r[11]};
    for (int i = 0; i < nx; i++) {
        const double *xi = x + 3 * i;
        const double dx[3] = {xi[0] - r[0], xi[1] - r[1], xi[2] - r[2]};
        const double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        if (rw > 0.0 && r2 > rw * rw) continue;
        const double ph = r[3] * dx[0] + r[4] * dx[1] + r[5] * dx[2];
        const cplx E = cexp(I * k * ph - 0.5 * k * r2);
        const cplx *u = ub + (size_t)i * 3;
        cplx Eb = 0;
        for (int d = 0; d < 3; d++) {
            Ab[d] += conj(E) * u[d];
            Eb += conj(A[d]) * u[d];
        }
        const cplx phb = conj(E) * Eb; /* d phi/d P = i k dx, d phi/d Q = -i k P + k dx */
        for (int d = 0; d < 3; d++) {
            Pb[d] += creal(conj(I * k * dx[d]) * phb);
            Qb[d] += creal(conj(-I * k * r[3 + d] + k * dx[d]) * phb);
        }
    }
    for (int d = 0; d < 3; d++) {
        rb[d] += Qb[d];
        rb[3 + d] += Pb[d];
        rb[6 + 2 * d] += creal(Ab[d]);
        rb[7 + 2 * d] += cimag(Ab[d]);
    }
}

/* adjoint of make_record (frame or scalar form): record cotangent rb -> cotangents of y0, f0, y1, f1 */
static void make_record_vjp(int mt, const orc_state *y0, const orc_state *f0, const orc_state *y1,
                            const orc_state *f1, double dt, double th, double w, const double rb[12], orc_state *y0b,
                            orc_state *f0b, orc_state *y1b, orc_state *f1b)
{
    const double h00 = 2 * th * th * th - 3 * th * th + 1, h10 = th * th * th - 2 * th * th + th;
    const double h01 = -2 * th * th * th + 3 * th * th, h11 = th * th * th - th * th;
    double P[3], Pb[3];
    for (int d = 0; d < 3; d++) {
        P[d] = h00 * y0->P[d] + h10 * dt * f0->P[d] + h01 * y1->P[d] + h11 * dt * f1->P[d];
        Pb[d] = rb[3 + d];
    }
    cplx a[3], ab[3] = {0, 0, 0};
    for (int j = 0; j < 3; j++) a[j] = (1.0 - th) * y0->a[j] + th * y1->a[j];
    const cplx Ab[3] = {rb[6] + I * rb[7], rb[8] + I * rb[9], rb[10] + I * rb[11]};
    const int cls = META_CLS(mt);
    if (cls < 2) {
        const double pn = norm3(P);
        double Ph[3], Phb[3];
        for (int d = 0; d < 3; d++) Ph[d] = P[d] / pn;
        for (int d = 0; d < 3; d++) {
            ab[0] += w * Ph[d] * Ab[d];
            Phb[d] = creal(conj(w * a[0]) * Ab[d]);
        }
        const double s = Ph[0] * Phb[0] + Ph[1] * Phb[1] + Ph[2] * Phb[2];
        for (int d = 0; d < 3; d++) Pb[d] += (Phb[d] - Ph[d] * s) / pn;
    } else if (!(mt & META_VECTOR)) {
        double Nsv[3], Nsh[3], Nsvb[3], Nshb[3];
        s_frame(P, (mt & META_REF_E1) != 0, Nsv, Nsh, NULL);
        for (int d = 0; d < 3; d++) {
            ab[0] += w * Nsv[d] * Ab[d];
            ab[1] += w * Nsh[d] * Ab[d];
            Nsvb[d] = creal(conj(w * a[0]) * Ab[d]);
            Nshb[d] = creal(conj(w * a[1]) * Ab[d]);
        }
        s_frame_vjp(P, (mt & META_REF_E1) != 0, Nsvb, Nshb, Pb);
    } else {
        for (int d = 0; d < 3; d++) ab[d] = w * Ab[d];
    }
    for (int j = 0; j < 3; j++) {
        y0b->a[j] += (1.0 - th) * ab[j];
        y1b->a[j] += th * ab[j];
    }
    for (int d = 0; d < 3; d++) {
        y0b->Q[d] += h00 * rb[d];
        f0b->Q[d] += h10 * dt * rb[d];
        y1b->Q[d] += h01 * rb[d];
        f1b->Q[d] += h11 * dt * rb[d];
        y0b->P[d] += h00 * Pb[d];
        f0b->P[d] += h10 * dt * Pb[d];
        y1b->P[d] += h01 * Pb[d];
        f1b->P[d] += h11 * dt * Pb[d];
    }
}

static void state_axpy_inplace(orc_state *o, double h, const orc_state *d)
{
    double *oo = (double *)o;
    const double *dd = (const double *)d;
    for (int i = 0; i < 48; i++) oo[i] += h * dd[i];
}

static int state_is_zero(const orc_state *s)
{
    const double *v = (const double *)s;
    for (int i = 0; i < 48; i++)
        if (v[i] != 0.0) return 0;
    return 1;
}

/* adjoint of rk4_step: given yb1 (cotangent of y_{n+1}) and an extra cotangent on k1 = f(y_n),
 * add the cotangent of y_n to yb0 and the model cotangents to gp/gs */
static void rk4_step_vjp(const orc_model *m, int mt, const orc_state *y, double dt, const orc_state *yb1,
                         const orc_state *k1b_extra, orc_state *yb0, double *gp, double *gs)
{
    orc_state k1, k2, k3, y2, y3, y4;
    orc_rhs(m, mt, y, &k1);
    axpy_state(&y2, y, 0.5 * dt, &k1);
    orc_rhs(m, mt, &y2, &k2);
    axpy_state(&y3, y, 0.5 * dt, &k2);
    orc_rhs(m, mt, &y3, &k3);
    axpy_state(&y4, y, dt, &k3);
    orc_state k1b, k2b, k3b, k4b, sb;
    memset(&k1b, 0, sizeof k1b);
    memset(&k2b, 0, sizeof k2b);
    memset(&k3b, 0, sizeof k3b);
    memset(&k4b, 0, sizeof k4b);
    state_axpy_inplace(yb0, 1.0, yb1);
    state_axpy_inplace(&k1b, dt / 6.0, yb1);
    state_axpy_inplace(&k2b, dt / 3.0, yb1);
    state_axpy_inplace(&k3b, dt / 3.0, yb1);
    state_axpy_inplace(&k4b, dt / 6.0, yb1);
    if (k1b_extra) state_axpy_inplace(&k1b, 1.0, k1b_extra);
    /* k4 = f(y + dt k3) */
    memset(&sb, 0, sizeof sb);
    orc_rhs_vjp(m, mt, &y4, &k4b, &sb, gp, gs);
    state_axpy_inplace(yb0, 1.0, &sb);
    state_axpy_inplace(&k3b, dt, &sb);
    /* k3 = f(y + dt/2 k2) */
    memset(&sb, 0, sizeof sb);
    orc_rhs_vjp(m, mt, &y3, &k3b, &sb, gp, gs);
    state_axpy_inplace(yb0, 1.0, &sb);
    state_axpy_inplace(&k2b, 0.5 * dt, &sb);
    /* k2 = f(y + dt/2 k1) */
    memset(&sb, 0, sizeof sb);
    orc_rhs_vjp(m, mt, &y2, &k2b, &sb, gp, gs);
    state_axpy_inplace(yb0, 1.0, &sb);
    state_axpy_inplace(&k1b, 0.5 * dt, &sb);
    /* k1 = f(y) */
    orc_rhs_vjp(m, mt, y, &k1b, yb0, gp, gs);
}

/* Reverse mode of orc_propagate + records + Gaussian sums at the nx points x for every sample:
 * u_j(x) = sum_b rec_jb(x).  Given the cotangents ub [ns][nx][3] (complex; dL/dRe u + i dL/dIm u)
 * writes the cotangent of each beam's initial state to stb [nb][48] and adds the model cotangents
 * (node fields of the P and S grids) to gp/gs (may be NULL).  Every trajectory is stored in full. */
int orc_solve_vjp(const orc_model *m, int nb, const double *st_, const int *meta, double dt, int nsteps, int ns,
                  const int *s_step, const double *s_theta, double w, double k, double rw, int nx, const double *x,
                  const double *ub_, double *stb_, double *gp, double *gs)
{
    const orc_state *st = (const orc_state *)st_;
    const cplx *ub = (const cplx *)ub_;
    orc_state *stb = (orc_state *)stb_;
    for (int b = 0; b < nb; b++)
        if ((meta[b] & META_VECTOR) || m->kind == ORC_LAYERED) return -1;
    int bad = 0;
#pragma omp parallel
    {
        orc_state *Y = (orc_state *)malloc(sizeof(orc_state) * (size_t)(nsteps + 1));
        orc_state *Fv = (orc_state *)malloc(sizeof(orc_state) * (size_t)(nsteps + 1));
        if (!Y || !Fv) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int b = 0; b < nb; b++) {
            if (!Y || !Fv) continue;
            const int mt = meta[b];
            Y[0] = st[b];
            orc_rhs(m, mt, &Y[0], &Fv[0]);
            for (int n = 0; n < nsteps; n++) {
                rk4_step(m, mt, &Y[n], &Fv[n], dt, &Y[n + 1]);
                orc_rhs(m, mt, &Y[n + 1], &Fv[n + 1]);
            }
            orc_state yb1;
            memset(&yb1, 0, sizeof yb1);
            int j = ns - 1;
            for (int n = nsteps - 1; n >= 0; n--) {
                orc_state y0b, f0b, f1b;
                memset(&y0b, 0, sizeof y0b);
                memset(&f0b, 0, sizeof f0b);
                memset(&f1b, 0, sizeof f1b);
                for (; j >= 0 && s_step[j] == n; j--) {
                    double rec[12], rb[12] = {0};
                    make_record(mt, &Y[n], &Fv[n], &Y[n + 1], &Fv[n + 1], dt, s_theta[j], w, rec);
                    gauss_vjp_record(rec, k, rw, nx, x, ub + (size_t)j * nx * 3, rb);
                    make_record_vjp(mt, &Y[n], &Fv[n], &Y[n + 1], &Fv[n + 1], dt, s_theta[j], w, rb, &y0b, &f0b,
                                    &yb1, &f1b);
                }
                if (!state_is_zero(&f1b)) orc_rhs_vjp(m, mt, &Y[n + 1], &f1b, &yb1, gp, gs);
                rk4_step_vjp(m, mt, &Y[n], dt, &yb1, &f0b, &y0b, gp, gs);
                yb1 = y0b;
            }
            stb[b] = yb1;
        }
        free(Y);
        free(Fv);
    }
    return bad ? -2 : 0;
}

/* Reverse mode of orc_beam_init with respect to the model: a = 2^{3/2} (F.n +- i G.n/(k c(q) |p|))/2
 * depends on the model only through c(q) in the G term.  Given the initial-state cotangents stb
 * (mesh order, one class) adds dL/dc(q) to the node fields through the interpolation weights. */
void orc_beam_init_vjp(const orc_model *m, double k, int nq, const double q0[3], const double dq[3], int np,
                       const double p0[3], const double dp[3], const double *F_, const double *G_, int cls,
                       const double *stb_, double *gp, double *gs)
{
    (void)F_;
    if (!G_) return;
    const cplx *G = (const cplx *)G_;
    const orc_state *stb = (const orc_state *)stb_;
    const long NP = (long)np * np * np;
    const long M = (long)nq * nq * nq * NP;
    const int wave = cls >= 2;
    const double sgn = (cls & 1) ? -1.0 : 1.0;
    for (long mi = 0; mi < M; mi++) {
        long iq = mi / NP, ip = mi % NP;
        int qi[3] = {(int)(iq / ((long)nq * nq)), (int)((iq / nq) % nq), (int)(iq % nq)};
        int pj[3] = {(int)(ip / ((long)np * np)), (int)((ip / np) % np), (int)(ip % np)};
        double q[3], p[3];
        for (int d = 0; d < 3; d++) {
            q[d] = q0[d] + qi[d] * dq[d];
            p[d] = p0[d] + pj[d] * dp[d];
        }
        const double pn = norm3(p);
        double cf[10];
        orc_model_eval(m, wave, q, cf);
        double dirs[2][3];
        int ndir;
        if (!wave) {
            for (int d = 0; d < 3; d++) dirs[0][d] = p[d] / pn;
            ndir = 1;
        } else {
            s_frame(p, orc_s_ref_e1(p), dirs[0], dirs[1], NULL);
            ndir = 2;
        }
        double cb = 0.0;
        for (int j = 0; j < ndir; j++) {
            cplx gn = 0;
            for (int d = 0; d < 3; d++) gn += G[mi * 3 + d] * dirs[j][d];
            /* d a_j / d c = -2^{3/2} (1/2) sgn i G.n / (k c^2 |p|) */
            const cplx da = -pow(2.0, 1.5) * 0.5 * sgn * I * gn / (k * cf[0] * cf[0] * pn);
            cb += creal(conj(da) * stb[mi].a[j]);
        }
        double cbar[10] = {cb, 0, 0, 0, 0, 0, 0, 0, 0, 0}, qb[3] = {0, 0, 0};
        model_vjp(m, wave, q, cbar, qb, gp, gs);
    }
}
