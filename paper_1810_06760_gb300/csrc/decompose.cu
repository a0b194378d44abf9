// A1-A2: wave-packet (FBI) transform of the initial data (Eq. psi) as three per-axis complex
// contractions, then beam initialisation (Eqs. alpha^k, ini_plus/ini_minus, op_zZ_app).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "fga_beam.cuh"

namespace fga {

// per-axis kernel K[a][i] = exp(-i k p (y_i - q) - k (y_i - q)^2 / 2), a = iq * np + jp
template <typename R>
__global__ void fbi_axis_kernel(C2<R> *__restrict__ K, int nq, int np, int ny, double q0, double dq, double p0,
                                double dp, double y0, double dy, double k) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int A = nq * np;
    if (idx >= A * ny) return;
    const int a = idx / ny, i = idx % ny;
    const int iq = a / np, jp = a % np;
    const double q = q0 + iq * dq, p = p0 + jp * dp, y = y0 + i * dy;
    const double d = y - q;
    double s, c;
    sincos(-k * p * d, &s, &c);
    const double e = exp(-0.5 * k * d * d);
    K[idx] = {(R)(e * c), (R)(e * s)};
}

template <typename R> __device__ __forceinline__ C2<R> to_c2(const double2 v) { return {(R)v.x, (R)v.y}; }
template <typename R> __device__ __forceinline__ C2<R> to_c2(const C2<R> v) { return v; }

// Batched strided complex GEMM: C[z][m][n] = scale * sum_k A[z][m][k] B[n][k].
// A elements of type TA (complex128 input or R intermediates), B and C of type R.
template <typename R, typename TA>
__global__ void __launch_bounds__(256) cgemm_kernel(const TA *__restrict__ A, int64_t sAz, int64_t sAm, int64_t sAk,
                                                    const C2<R> *__restrict__ B, int64_t sBn, int64_t sBk,
                                                    C2<R> *__restrict__ Cm, int64_t sCz, int64_t sCm, int64_t sCn,
                                                    int64_t M, int N, int K, R scale) {
    constexpr int TM = 64, TN = 64, TK = 16;
    __shared__ C2<R> As[TK][TM + 1];
    __shared__ C2<R> Bs[TK][TN + 1];
    const int z = blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    C2<R> acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = {R(0), R(0)};
    const TA *Az = A + z * sAz;
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = threadIdx.x; e < TK * TM; e += 256) {
            const int mm = e % TM, kk = e / TM;
            const int64_t gm = m0 + mm;
            const int gk = k0 + kk;
            C2<R> v = {R(0), R(0)};
            if (gm < M && gk < K) v = to_c2<R>(Az[gm * sAm + (int64_t)gk * sAk]);
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            const int nn = e % TN, kk = e / TN;
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < K) ? B[(int64_t)gn * sBn + (int64_t)gk * sBk] : C2<R>{R(0), R(0)};
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            C2<R> a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    acc[i][j].r += a[i].r * b[j].r - a[i].i * b[j].i;
                    acc[i][j].i += a[i].r * b[j].i + a[i].i * b[j].r;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t gm = m0 + tx + 16 * i;
            const int gn = n0 + ty + 16 * j;
            if (gm < M && gn < N)
                Cm[z * sCz + gm * sCm + (int64_t)gn * sCn] = {acc[i][j].r * scale, acc[i][j].i * scale};
        }
}

template <typename R, typename TA>
static fga_status cgemm(const TA *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<R> *B, int64_t sBn, int64_t sBk,
                        C2<R> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z, int64_t M, int N, int K, R scale,
                        cudaStream_t s) {
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((N + 63) / 64), (unsigned)Z);
    ProfScope ps(P_DECOMP, s);
    cgemm_kernel<R, TA><<<grid, 256, 0, s>>>(A, sAz, sAm, sAk, B, sBn, sBk, Cm, sCz, sCm, sCn, M, N, K, scale);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

// F[a0][a1][a2][c] = dy^3 sum_y f[y0][y1][y2][c] K0[a0][y0] K1[a1][y1] K2[a2][y2]
// The three stages (contract y2, then y1, then y0) are batched strided complex GEMMs: on the tensor
// cores (FP16 split, FP32 accumulation) for the FP32 path, on the FP64 pipe for the FP64 path.
struct TransformScratch {
    float *amax = nullptr;   // DEVICE: max |Re|, |Im| of the input
    int *err = nullptr;      // DEVICE: set by a tensor-core wait that ran out
    double S[3] = {1, 1, 1}; // max over kernel rows of sum_i |K_d[a][i]| per axis (bounds of the stages)
};

template <typename R>
static fga_status stage_gemm(const double2 *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<R> *B, int64_t sBn,
                             int64_t sBk, C2<R> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z, int64_t M, int N,
                             int K, R scale, const TransformScratch &ts, double factor, cudaStream_t s);
template <typename R>
static fga_status stage_gemm(const C2<R> *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<R> *B, int64_t sBn,
                             int64_t sBk, C2<R> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z, int64_t M, int N,
                             int K, R scale, const TransformScratch &ts, double factor, cudaStream_t s);

template <>
fga_status stage_gemm<double>(const double2 *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<double> *B,
                              int64_t sBn, int64_t sBk, C2<double> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z,
                              int64_t M, int N, int K, double scale, const TransformScratch &, double, cudaStream_t s) {
    return cgemm<double, double2>(A, sAz, sAm, sAk, B, sBn, sBk, Cm, sCz, sCm, sCn, Z, M, N, K, scale, s);
}
template <>
fga_status stage_gemm<double>(const C2<double> *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<double> *B,
                              int64_t sBn, int64_t sBk, C2<double> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z,
                              int64_t M, int N, int K, double scale, const TransformScratch &, double, cudaStream_t s) {
    return cgemm<double, C2<double>>(A, sAz, sAm, sAk, B, sBn, sBk, Cm, sCz, sCm, sCn, Z, M, N, K, scale, s);
}
template <>
fga_status stage_gemm<float>(const double2 *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<float> *B, int64_t sBn,
                             int64_t sBk, C2<float> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z, int64_t M, int N,
                             int K, float scale, const TransformScratch &ts, double factor, cudaStream_t s) {
    return tc_cgemm<double2>(A, sAz, sAm, sAk, reinterpret_cast<const float2 *>(B), sBn, sBk,
                             reinterpret_cast<float2 *>(Cm), sCz, sCm, sCn, Z, M, N, K, scale, ts.amax, (float)factor,
                             ts.err, s);
}
template <>
fga_status stage_gemm<float>(const C2<float> *A, int64_t sAz, int64_t sAm, int64_t sAk, const C2<float> *B,
                             int64_t sBn, int64_t sBk, C2<float> *Cm, int64_t sCz, int64_t sCm, int64_t sCn, int Z,
                             int64_t M, int N, int K, float scale, const TransformScratch &ts, double factor,
                             cudaStream_t s) {
    return tc_cgemm<float2>(reinterpret_cast<const float2 *>(A), sAz, sAm, sAk, reinterpret_cast<const float2 *>(B),
                            sBn, sBk, reinterpret_cast<float2 *>(Cm), sCz, sCm, sCn, Z, M, N, K, scale, ts.amax,
                            (float)factor, ts.err, s);
}

template <typename R>
static fga_status fbi_transform(const fga_init_desc *d, const double2 *f, C2<R> *const Kax[3], C2<R> *T1, C2<R> *T2,
                                C2<R> *F, const TransformScratch &ts, cudaStream_t s) {
    const int A = d->nq * d->np;
    const int n0 = d->ny[0], n1 = d->ny[1], n2 = d->ny[2];
    if (sizeof(R) == 4) FGA_TRY(tc_absmax(f, (int64_t)n0 * n1 * n2 * 3, ts.amax, s));
    // |Re|, |Im| of a stage's output <= sqrt(2) max(|Re|, |Im|) of its input x sum_i |K[a][i]|
    const double g1 = std::sqrt(2.0) * ts.S[2], g2 = g1 * std::sqrt(2.0) * ts.S[1];
    // stage 1 (contract y2), one GEMM per component c: T1[(y0,y1)][a2][c]
    FGA_TRY((stage_gemm<R>(f, 1, (int64_t)n2 * 3, 3, Kax[2], n2, 1, T1, 1, (int64_t)A * 3, 3, 3, (int64_t)n0 * n1, A,
                           n2, R(1), ts, 1.0, s)));
    // stage 2 (contract y1): T2[y0][a1][(a2,c)] ; batch y0, m = (a2,c), n = a1, k = y1
    FGA_TRY((stage_gemm<R>((const C2<R> *)T1, (int64_t)n1 * A * 3, 1, (int64_t)A * 3, Kax[1], n1, 1, T2,
                           (int64_t)A * A * 3, 1, (int64_t)A * 3, n0, (int64_t)A * 3, A, n1, R(1), ts, g1, s)));
    // stage 3 (contract y0): F[a0][(a1,a2,c)], m = (a1,a2,c), n = a0, k = y0
    const R vol = (R)(d->dy[0] * d->dy[1] * d->dy[2]);
    FGA_TRY((stage_gemm<R>((const C2<R> *)T2, 0, 1, (int64_t)A * A * 3, Kax[0], n0, 1, F, 0, 1, (int64_t)A * A * 3, 1,
                           (int64_t)A * A * 3, A, n0, vol, ts, g2, s)));
    return FGA_OK;
}

// max over the q nodes of sum_i exp(-k (y_i - q)^2 / 2): the largest row sum of |K| on one axis
static double kernel_row_sum_max(int nq, double q0, double dq, int ny, double y0, double dy, double k) {
    double best = 0.0;
    for (int iq = 0; iq < nq; iq++) {
        const double q = q0 + iq * dq;
        double sum = 0.0;
        for (int i = 0; i < ny; i++) {
            const double t = y0 + i * dy - q;
            sum += std::exp(-0.5 * k * t * t);
        }
        best = std::max(best, sum);
    }
    return best;
}

// initial state and flags of the beam of mesh point mi and class cls
template <typename R, int MED>
__device__ __forceinline__ void beam_init_state(const ModelDev &Md, const C2<R> *__restrict__ F,
                                                const C2<R> *__restrict__ G, int nq, int np, double3 q0, double3 dq,
                                                double3 p0, double3 dp, double k, int64_t mi, int cls, R *y, int &fl) {
    const int64_t NP = (int64_t)np * np * np;
    const int64_t iq = mi / NP, ip = mi % NP;
    const int qi[3] = {(int)(iq / ((int64_t)nq * nq)), (int)((iq / nq) % nq), (int)(iq % nq)};
    const int pj[3] = {(int)(ip / ((int64_t)np * np)), (int)((ip / np) % np), (int)(ip % np)};
    const double qd[3] = {q0.x + qi[0] * dq.x, q0.y + qi[1] * dq.y, q0.z + qi[2] * dq.z};
    const double pd[3] = {p0.x + pj[0] * dp.x, p0.y + pj[1] * dp.y, p0.z + pj[2] * dp.z};
    const int A = nq * np;
    const int64_t fidx = (((int64_t)(qi[0] * np + pj[0]) * A + (qi[1] * np + pj[1])) * A + (qi[2] * np + pj[2])) * 3;
    const int wave = cls >= 2;
    R q[3] = {(R)qd[0], (R)qd[1], (R)qd[2]};
    R p[3] = {(R)pd[0], (R)pd[1], (R)pd[2]};
    R cf[10];
    // layered media: the layer of q from its depth along the layer normal (x3 unless the layers are tilted),
    // minus its distance to the centre of spherical layers, or the undulating interfaces at or above it;
    // c(q) is that layer's speed
    int lay = 0;
    if (MED == FGA_MEDIUM_LAYERED) {
        if (Md.undul) {
            const double cc = cos(Md.uk[0] * qd[0]) * cos(Md.uk[1] * qd[1]);
            for (int l = 0; l < Md.nlay - 1; l++) lay += (qd[2] >= Md.zif[l] + Md.uamp[l] * cc) ? 1 : 0;
        } else {
            double zl = qd[2];
            if (Md.shells) {
                const double r0 = qd[0] - Md.ctr[0], r1 = qd[1] - Md.ctr[1], r2 = qd[2] - Md.ctr[2];
                zl = -sqrt(r0 * r0 + r1 * r1 + r2 * r2);
            } else if (Md.tilted) {
                zl = Md.R[6] * qd[0] + Md.R[7] * qd[1] + Md.R[8] * qd[2];
            }
            for (int l = 0; l < Md.nlay - 1; l++) lay += (zl >= Md.zif[l]) ? 1 : 0;
        }
        cf[0] = wave ? mp<R>(Md.lcs[lay], Md.flcs[lay]) : mp<R>(Md.lcp[lay], Md.flcp[lay]);
        for (int f = 1; f < 10; f++) cf[f] = R(0);
    } else {
        model_eval<R, MED>(Md, wave, q, cf);
    }
    const R pn = Real<R>::sqrt_(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const R sgn = (cls & 1) ? R(-1) : R(1);
    const R gsc = sgn / ((R)k * cf[0] * pn);  // +- 1/(k c(q) |p|)
    R dirs[2][3];
    int nd = 1;
    fl = cls;
    if (!wave) {
        for (int d = 0; d < 3; d++) dirs[0][d] = p[d] / pn;
    } else {
        const bool r1 = (p[0] * p[0] + p[1] * p[1]) < R(0.01) * pn * pn;
        if (r1) fl |= FL_REF_E1;
        s_frame<R>(p, r1, dirs[0], dirs[1]);
        nd = 2;
    }
    const R a0 = R(2.8284271247461900976033774484194);  // 2^{3/2}
    R amp[4] = {R(0), R(0), R(0), R(0)};
    for (int j = 0; j < nd; j++) {
        R fr = R(0), fi = R(0), gr = R(0), gi = R(0);
        for (int d = 0; d < 3; d++) {
            fr += F[fidx + d].r * dirs[j][d];
            fi += F[fidx + d].i * dirs[j][d];
            if (G) {
                gr += G[fidx + d].r * dirs[j][d];
                gi += G[fidx + d].i * dirs[j][d];
            }
        }
        // psi = (F.n +- i G.n / (k c |p|)) / 2
        amp[2 * j] = a0 * R(0.5) * (fr - gsc * gi);
        amp[2 * j + 1] = a0 * R(0.5) * (fi + gsc * gr);
    }
    if (MED == FGA_MEDIUM_LAYERED) fl |= (lay << 4) | (cls << FL_ROOT_SHIFT);
    for (int f = 0; f < NF; f++) y[f] = R(0);
    for (int d = 0; d < 3; d++) {
        y[F_Q + d] = q[d];
        y[F_P + d] = p[d];
        y[F_DQ + 2 * (3 * d + d)] = R(1);      // dzQ = I
        y[F_DP + 2 * (3 * d + d) + 1] = R(-1); // dzP = -i I
    }
    y[F_A0] = amp[0];
    y[F_A0 + 1] = amp[1];
    y[F_A1] = amp[2];
    y[F_A1 + 1] = amp[3];
}

// |psi|^2 of a beam from its initial amplitudes (2^{3/2} psi): the same value on every pass
template <typename R> __device__ __forceinline__ R psi_mag2(const R *y) {
    return y[F_A0] * y[F_A0] + y[F_A0 + 1] * y[F_A0 + 1] + y[F_A1] * y[F_A1] + y[F_A1 + 1] * y[F_A1 + 1];
}

// keep rule of the psi-threshold selection: |psi|^2 > eps^2 max|psi|^2 (amax2 holds the bits of the max)
template <typename R> struct MaxBits;
template <> struct MaxBits<float> {
    using U = unsigned;
    static __device__ U bits(float v) { return __float_as_uint(v); }
    static __device__ float val(U u) { return __uint_as_float(u); }
};
template <> struct MaxBits<double> {
    using U = unsigned long long;
    static __device__ U bits(double v) { return (U)__double_as_longlong(v); }
    static __device__ double val(U u) { return __longlong_as_double((long long)u); }
};

// one beam per (mesh point, requested class); with sel != NULL only the beams whose sel[mi] differs
// from sel[mi + 1] (an exclusive scan of the keep flags) are written, at off + sel[mi]
template <typename R, int MED>
__global__ void beam_init_kernel(ModelDev Md, const C2<R> *__restrict__ F, const C2<R> *__restrict__ G, int nq, int np,
                                 double3 q0, double3 dq, double3 p0, double3 dp, double k, int64_t M, int cls,
                                 int64_t off, int64_t cap, R *__restrict__ st, int32_t *__restrict__ flags,
                                 int32_t *__restrict__ ids, const uint32_t *__restrict__ sel) {
    const int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= M) return;
    if (sel && sel[mi + 1] == sel[mi]) return;
    R y[NF];
    int fl;
    beam_init_state<R, MED>(Md, F, G, nq, np, q0, dq, p0, dp, k, mi, cls, y, fl);
    const int64_t b = off + (sel ? (int64_t)sel[mi] : mi);
    for (int f = 0; f < NF; f++) st[(int64_t)f * cap + b] = y[f];
    flags[b] = fl;
    ids[b] = (int32_t)mi;
}

// tilted layered media: the beams of [0, nb) into the layer frame x' = R x (rows of R the frame's axes):
// Q, P rotate, each row m of dzQ and dzP (the vector dQ/dz_m) rotates, S amplitudes are re-expressed in
// the S frame of the rotated P (the polarisation vector a_sv N_sv + a_sh N_sh rotates with the beam)
template <typename R>
__global__ void rotate_to_layer_frame_kernel(ModelDev Md, R *__restrict__ st, int32_t *__restrict__ flags,
                                             int64_t nb, int64_t cap) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    R y[NF];
    for (int f = 0; f < NF; f++) y[f] = st[(int64_t)f * cap + b];
    int fl = flags[b];
    rotate_state<R>(Md.R, false, true, y, fl);
    flags[b] = fl;
    for (int f = 0; f < NF; f++) st[(int64_t)f * cap + b] = y[f];
}

// pass 1 of the selection: the largest |psi|^2 over the class (block maximum, one atomic per block)
template <typename R, int MED>
__global__ void __launch_bounds__(128) psi_max_kernel(ModelDev Md, const C2<R> *__restrict__ F,
                                                      const C2<R> *__restrict__ G, int nq, int np, double3 q0,
                                                      double3 dq, double3 p0, double3 dp, double k, int64_t M, int cls,
                                                      typename MaxBits<R>::U *__restrict__ amax2) {
    const int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    R m2 = R(0);
    if (mi < M) {
        R y[NF];
        int fl;
        beam_init_state<R, MED>(Md, F, G, nq, np, q0, dq, p0, dp, k, mi, cls, y, fl);
        m2 = psi_mag2<R>(y);
        if (!(m2 == m2)) m2 = R(0);   // a NaN amplitude is reported by the solve, not selected on
    }
    for (int o = 16; o; o >>= 1) m2 = max(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    __shared__ R wm[4];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        const R b = max(max(wm[0], wm[1]), max(wm[2], wm[3]));
        atomicMax(amax2, MaxBits<R>::bits(b));
    }
}

// pass 2: keep[mi] = 1 for |psi|^2 > eps2 * max|psi|^2, keep[M] = 0 (room for the scan's total); the
// class's survivor count is added to *count
template <typename R, int MED>
__global__ void __launch_bounds__(128) psi_keep_kernel(ModelDev Md, const C2<R> *__restrict__ F,
                                                       const C2<R> *__restrict__ G, int nq, int np, double3 q0,
                                                       double3 dq, double3 p0, double3 dp, double k, int64_t M,
                                                       int cls, const typename MaxBits<R>::U *__restrict__ amax2,
                                                       R eps2, uint32_t *__restrict__ keep,
                                                       unsigned long long *__restrict__ count) {
    const int64_t mi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned kf = 0;
    if (mi < M) {
        R y[NF];
        int fl;
        beam_init_state<R, MED>(Md, F, G, nq, np, q0, dq, p0, dp, k, mi, cls, y, fl);
        const R lim = eps2 * MaxBits<R>::val(*amax2);
        kf = psi_mag2<R>(y) > lim ? 1u : 0u;
        keep[mi] = kf;
    } else if (mi == M) {
        keep[M] = 0u;
    }
    const unsigned n = __popc(__ballot_sync(0xffffffffu, kf));
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, (unsigned long long)n);
}

// F (and G from g, if both are given) = the transform of Eq. psi in the per-axis pair layout
// [a0][a1][a2][3], a_d = iq_d * np + jp_d.  Synchronises s before its temporaries are released; reports
// a tensor-core wait that ran out as FGA_ERR_TIMEOUT.
template <typename R>
static fga_status transform_typed(const fga_init_desc *d, const double2 *f, const double2 *g, C2<R> *F, C2<R> *G,
                                  cudaStream_t s) {
    const int A = d->nq * d->np;
    ScopedDevBuf Kb, T1, T2, tsb;
    const size_t kbytes = sizeof(C2<R>) * (size_t)A * (d->ny[0] + d->ny[1] + d->ny[2]);
    FGA_TRY(Kb.ensure(kbytes));
    C2<R> *Kax[3];
    Kax[0] = Kb.as<C2<R>>();
    Kax[1] = Kax[0] + (size_t)A * d->ny[0];
    Kax[2] = Kax[1] + (size_t)A * d->ny[1];
    for (int ax = 0; ax < 3; ax++) {
        const int tot = A * d->ny[ax];
        ProfScope ps(P_DECOMP, s);
        fbi_axis_kernel<R><<<(tot + 255) / 256, 256, 0, s>>>(Kax[ax], d->nq, d->np, d->ny[ax], d->q0[ax], d->dq[ax],
                                                            d->p0[ax], d->dp[ax], d->y0[ax], d->dy[ax], d->k);
    }
    FGA_CUDA(cudaGetLastError());
    FGA_TRY(T1.ensure(sizeof(C2<R>) * (size_t)d->ny[0] * d->ny[1] * A * 3));
    FGA_TRY(T2.ensure(sizeof(C2<R>) * (size_t)d->ny[0] * A * A * 3));
    FGA_TRY(tsb.ensure(64));
    TransformScratch ts;
    ts.amax = tsb.as<float>();
    ts.err = reinterpret_cast<int *>(tsb.as<char>() + 16);
    FGA_CUDA(cudaMemsetAsync(tsb.p, 0, 64, s));
    for (int a = 0; a < 3; a++)
        ts.S[a] = kernel_row_sum_max(d->nq, d->q0[a], d->dq[a], d->ny[a], d->y0[a], d->dy[a], d->k);
    FGA_TRY(fbi_transform<R>(d, f, Kax, T1.as<C2<R>>(), T2.as<C2<R>>(), F, ts, s));
    if (g && G) FGA_TRY(fbi_transform<R>(d, g, Kax, T1.as<C2<R>>(), T2.as<C2<R>>(), G, ts, s));
    // the temporaries are released when this scope ends; make sure the stream is done with them
    FGA_CUDA(cudaStreamSynchronize(s));
    if (sizeof(R) == 4) {
        int terr = 0;
        FGA_CUDA(cudaMemcpy(&terr, ts.err, sizeof terr, cudaMemcpyDeviceToHost));
        if (terr) {
            set_error("wave-packet transform: a tensor-core wait ran out");
            return FGA_ERR_TIMEOUT;
        }
    }
    return FGA_OK;
}

// Beam-set storage for the class counts in b->n_cls: class blocks in class order, capacity rounded
// to 32 (layered media: growth x the initial count, for the children created at interfaces)
static fga_status beams_allocate(fga_beams *b, const fga_init_desc *d, cudaStream_t s) {
    int64_t off = 0;
    for (int c = 0; c < 4; c++) {
        b->off_cls[c] = off;
        off += b->n_cls[c];
    }
    b->nb = off;
    if (b->layered) {
        const double growth = d->growth > 0 ? std::max(1.0, d->growth) : 4.0;
        b->cap = ((int64_t)std::ceil(growth * (double)off) + 31) / 32 * 32;
    } else {
        b->cap = (off + 31) / 32 * 32;
    }
    b->cap = std::max<int64_t>(b->cap, 32);
    const size_t rb = d->precision == FGA_PREC_FP64 ? 8 : 4;
    FGA_TRY(b->state.ensure(rb * NFS * b->cap));
    // the Q compensation starts at zero
    FGA_CUDA(cudaMemsetAsync(static_cast<char *>(b->state.p) + rb * F_QC * b->cap, 0, rb * 3 * b->cap, s));
    FGA_TRY(b->flags.ensure(4 * b->cap));
    FGA_TRY(b->id.ensure(4 * b->cap));
    if (b->layered) {
        FGA_TRY(b->path.ensure(8 * b->cap));
        FGA_TRY(b->counts.ensure(16));
        FGA_TRY(b->n_begin.ensure(8));
        const unsigned long long c0[2] = {(unsigned long long)off, 0ull};
        FGA_CUDA(cudaMemsetAsync(b->path.p, 0, 8 * b->cap, s));
        FGA_CUDA(cudaMemcpyAsync(b->counts.p, c0, sizeof c0, cudaMemcpyHostToDevice, s));
        FGA_CUDA(cudaStreamSynchronize(s));
    }
    return FGA_OK;
}

template <typename R, int MED>
static fga_status decompose_medium(const fga_model *m, const fga_init_desc *d, fga_beams *b, const C2<R> *F,
                                   const C2<R> *G, cudaStream_t s) {
    const int64_t M = (int64_t)d->nq * d->nq * d->nq * d->np * d->np * d->np;
    const double3 q0 = {d->q0[0], d->q0[1], d->q0[2]}, dq = {d->dq[0], d->dq[1], d->dq[2]};
    const double3 p0 = {d->p0[0], d->p0[1], d->p0[2]}, dp = {d->dp[0], d->dp[1], d->dp[2]};
    const bool select = d->psi_rel_min > 0;
    using U = typename MaxBits<R>::U;
    ScopedDevBuf keepb, selb;
    U *amax2 = nullptr;
    unsigned long long *cnt = nullptr;
    uint32_t *keep = nullptr;
    const R eps2 = (R)(d->psi_rel_min * d->psi_rel_min);
    const unsigned kblocks = (unsigned)((M + 1 + 127) / 128);
    if (select) {
        // Step 1 of Fig. fig:FGA_alg chooses the beams worth propagating: |psi| > eps max|psi|, the maximum
        // over every requested class and mesh point
        FGA_TRY(selb.ensure(64));
        amax2 = selb.as<U>();
        cnt = reinterpret_cast<unsigned long long *>(selb.as<char>() + 16);
        FGA_CUDA(cudaMemsetAsync(selb.p, 0, 64, s));
        FGA_TRY(keepb.ensure(sizeof(uint32_t) * (size_t)(M + 1)));
        keep = keepb.as<uint32_t>();
        for (int cls = 0; cls < 4; cls++) {
            if (!(d->class_mask & (1u << cls))) continue;
            ProfScope ps(P_DECOMP, s);
            psi_max_kernel<R, MED><<<(unsigned)((M + 127) / 128), 128, 0, s>>>(m->dev, F, G, d->nq, d->np, q0, dq, p0,
                                                                              dp, d->k, M, cls, amax2);
        }
        FGA_CUDA(cudaGetLastError());
        for (int cls = 0; cls < 4; cls++) {
            if (!(d->class_mask & (1u << cls))) continue;
            ProfScope ps(P_DECOMP, s);
            psi_keep_kernel<R, MED><<<kblocks, 128, 0, s>>>(m->dev, F, G, d->nq, d->np, q0, dq, p0, dp, d->k, M, cls,
                                                            amax2, eps2, keep, cnt + cls);
        }
        FGA_CUDA(cudaGetLastError());
        unsigned long long hc[4];
        FGA_CUDA(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
        FGA_CUDA(cudaStreamSynchronize(s));
        int64_t tot = 0;
        for (int c = 0; c < 4; c++) {
            b->n_cls[c] = (d->class_mask & (1u << c)) ? (int64_t)hc[c] : 0;
            tot += b->n_cls[c];
        }
        FGA_CHECK(tot < (int64_t)1 << 31, "fga_decompose: more than 2^31 selected beams");
    } else {
        for (int c = 0; c < 4; c++) b->n_cls[c] = (d->class_mask & (1u << c)) ? M : 0;
    }
    FGA_TRY(beams_allocate(b, d, s));
    for (int cls = 0; cls < 4; cls++) {
        if (!b->n_cls[cls]) continue;
        if (select) {
            {
                ProfScope ps(P_DECOMP, s);
                psi_keep_kernel<R, MED><<<kblocks, 128, 0, s>>>(m->dev, F, G, d->nq, d->np, q0, dq, p0, dp, d->k, M,
                                                                cls, amax2, eps2, keep, cnt + 4);
            }
            FGA_CUDA(cudaGetLastError());
            FGA_TRY(scan_exclusive_u32(keep, M + 1, s));
        }
        ProfScope ps(P_DECOMP, s);
        beam_init_kernel<R, MED><<<(unsigned)((M + 127) / 128), 128, 0, s>>>(
            m->dev, F, G, d->nq, d->np, q0, dq, p0, dp, d->k, M, cls, b->off_cls[cls], b->cap, b->state.as<R>(),
            b->flags.as<int32_t>(), b->id.as<int32_t>(), select ? keep : nullptr);
        FGA_CUDA(cudaGetLastError());
    }
    if (MED == FGA_MEDIUM_LAYERED && m->dev.tilted) {
        b->tilted = true;
        for (int i = 0; i < 9; i++) b->R[i] = m->dev.R[i];
        if (b->nb > 0) {
            ProfScope ps(P_DECOMP, s);
            rotate_to_layer_frame_kernel<R><<<(unsigned)((b->nb + 127) / 128), 128, 0, s>>>(
                m->dev, b->state.as<R>(), b->flags.as<int32_t>(), b->nb, b->cap);
        }
        FGA_CUDA(cudaGetLastError());
    }
    // the selection scratch is released when this scope ends
    FGA_CUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

template <typename R>
static fga_status decompose_typed(const fga_model *m, const fga_init_desc *d, fga_beams *b, cudaStream_t s) {
    const int A = d->nq * d->np;
    ScopedDevBuf Fb, Gb;
    const size_t Fn = (size_t)A * A * A * 3;
    FGA_TRY(Fb.ensure(sizeof(C2<R>) * Fn));
    const C2<R> *G = nullptr;
    if (d->g) {
        FGA_TRY(Gb.ensure(sizeof(C2<R>) * Fn));
        G = Gb.as<C2<R>>();
    }
    FGA_TRY(transform_typed<R>(d, static_cast<const double2 *>(d->f), static_cast<const double2 *>(d->g),
                               Fb.as<C2<R>>(), Gb.as<C2<R>>(), s));
    const C2<R> *F = Fb.as<C2<R>>();
    switch (m->dev.kind) {
    case FGA_MEDIUM_CONST: FGA_TRY((decompose_medium<R, FGA_MEDIUM_CONST>(m, d, b, F, G, s))); break;
    case FGA_MEDIUM_SINE: FGA_TRY((decompose_medium<R, FGA_MEDIUM_SINE>(m, d, b, F, G, s))); break;
    case FGA_MEDIUM_GRID: FGA_TRY((decompose_medium<R, FGA_MEDIUM_GRID>(m, d, b, F, G, s))); break;
    default: FGA_TRY((decompose_medium<R, FGA_MEDIUM_LAYERED>(m, d, b, F, G, s))); break;
    }
    // F and G are released when this scope ends; make sure the stream is done with them
    FGA_CUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

fga_status decompose_impl(const fga_model *m, const fga_init_desc *d, fga_beams **out, cudaStream_t s) {
    FGA_CHECK(m && d && out, "fga_decompose: NULL argument");
    FGA_CHECK(std::isfinite(d->k) && d->k > 0, "fga_decompose: k must be > 0");
    FGA_CHECK(d->f != nullptr, "fga_decompose: f is NULL");
    FGA_CHECK(d->nq >= 1 && d->np >= 1, "fga_decompose: nq, np must be >= 1");
    FGA_CHECK(d->ny[0] >= 1 && d->ny[1] >= 1 && d->ny[2] >= 1, "fga_decompose: ny must be >= 1");
    FGA_CHECK((d->class_mask & 15u) != 0 && (d->class_mask & ~15u) == 0, "fga_decompose: class_mask must be in 1..15");
    FGA_CHECK(d->precision == FGA_PREC_FP32 || d->precision == FGA_PREC_FP64, "fga_decompose: bad precision");
    FGA_CHECK(std::isfinite(d->psi_rel_min) && d->psi_rel_min >= 0 && d->psi_rel_min < 1,
              "fga_decompose: psi_rel_min must be in [0, 1)");
    for (int a = 0; a < 3; a++) FGA_CHECK(d->dy[a] > 0 && d->dq[a] > 0 && d->dp[a] > 0, "fga_decompose: spacings must be > 0");
    const int64_t M = (int64_t)d->nq * d->nq * d->nq * d->np * d->np * d->np;
    // mesh indices are int32; without a selection every mesh point of every class is a beam slot
    FGA_CHECK(M < (int64_t)1 << 31, "fga_decompose: more than 2^31 mesh points");
    if (!(d->psi_rel_min > 0)) {
        int nc = 0;
        for (int c = 0; c < 4; c++) nc += (d->class_mask >> c) & 1;
        FGA_CHECK(M * nc < (int64_t)1 << 31, "fga_decompose: more than 2^31 beams");
    }
    fga_beams *b = new fga_beams();
    b->precision = d->precision;
    b->k = d->k;
    double vol = 1.0;
    for (int a = 0; a < 3; a++) vol *= d->dq[a] * d->dp[a];
    b->w = vol / std::pow(2.0 * M_PI / d->k, 4.5);
    b->layered = m->dev.kind == FGA_MEDIUM_LAYERED;
    if (b->layered) {
        b->gmax = d->max_interfaces > 0 ? d->max_interfaces : 4;
        b->rel_min = d->child_rel_min > 0 ? d->child_rel_min : 1e-6;
    }
    const fga_status st =
        d->precision == FGA_PREC_FP64 ? decompose_typed<double>(m, d, b, s) : decompose_typed<float>(m, d, b, s);
    if (st != FGA_OK) {
        fga_beams_destroy(b);
        return st;
    }
    b->last_stream = s;
    *out = b;
    return FGA_OK;
}

fga_status transform_impl(const fga_init_desc *d, void *F_out, cudaStream_t s) {
    FGA_CHECK(d && F_out, "fga_transform: NULL argument");
    FGA_CHECK(std::isfinite(d->k) && d->k > 0, "fga_transform: k must be > 0");
    FGA_CHECK(d->f != nullptr, "fga_transform: f is NULL");
    FGA_CHECK(d->nq >= 1 && d->np >= 1, "fga_transform: nq, np must be >= 1");
    FGA_CHECK(d->ny[0] >= 1 && d->ny[1] >= 1 && d->ny[2] >= 1, "fga_transform: ny must be >= 1");
    FGA_CHECK(d->precision == FGA_PREC_FP32 || d->precision == FGA_PREC_FP64, "fga_transform: bad precision");
    for (int a = 0; a < 3; a++) FGA_CHECK(d->dy[a] > 0 && d->dq[a] > 0 && d->dp[a] > 0, "fga_transform: spacings must be > 0");
    const int64_t A = (int64_t)d->nq * d->np;
    FGA_CHECK(A * A * A * 3 < (int64_t)1 << 31, "fga_transform: more than 2^31 output values");
    if (d->precision == FGA_PREC_FP64)
        return transform_typed<double>(d, static_cast<const double2 *>(d->f), nullptr, static_cast<C2<double> *>(F_out),
                                       nullptr, s);
    return transform_typed<float>(d, static_cast<const double2 *>(d->f), nullptr, static_cast<C2<float> *>(F_out),
                                  nullptr, s);
}

}  // namespace fga
