// Cross-correlation traveltime misfit and its adjoint source (the paper's inversion section applies
// FGA to wave-equation traveltime tomography after Tromp, Tape and Liu 2005; the paper itself prints
// no formula).  The adjoint source is a seismogram cotangent, so the gradient of the traveltime
// misfit is fga_solve_vjp fed with it.
//
// Per receiver r (one CTA): both records, [n_t][3] complex, are staged in shared memory as FP64; the
// correlation C(m) = sum_j sum_c Re(conj(s[j]) d[j+m]) for lags m = -M..M (one lag per thread at a
// time); the largest value, the smallest lag among equal values; a parabolic sub-sample step
// through the two neighbours; then N = (1/dt) sum |s[j+1] - s[j]|^2 (zero-padded ends) and the
// cotangent ubar[j] = tau (s[j+1] - s[j-1]) / (2 N) of the misfit 1/2 sum tau^2.  The correlation
// and the delay are FP64 whatever the record precision, so the integer lag is decided in the same
// precision as by a double-precision reference.  A second one-block kernel sums the misfit in a
// fixed order.
#include <cfloat>
#include <climits>
#include <cmath>

#include "fga_internal.cuh"

namespace fga {
namespace {

constexpr int TT_THREADS = 256;

__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ void put(float2 *p, double re, double im) { *p = make_float2((float)re, (float)im); }
__device__ __forceinline__ void put(double2 *p, double re, double im) { *p = make_double2(re, im); }

// block reduction of (value, lag): largest value, smallest lag among equal values
__device__ void argmax_block(double &v, int &m, double *sv, int *sm) {
    const int tid = threadIdx.x;
    sv[tid] = v;
    sm[tid] = m;
    __syncthreads();
    for (int o = TT_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) {
            const double w = sv[tid + o];
            const int l = sm[tid + o];
            if (w > sv[tid] || (w == sv[tid] && l < sm[tid])) {
                sv[tid] = w;
                sm[tid] = l;
            }
        }
        __syncthreads();
    }
    v = sv[0];
    m = sm[0];
    __syncthreads();
}

__device__ double sum_block(double v, double *sv) {
    const int tid = threadIdx.x;
    sv[tid] = v;
    __syncthreads();
    for (int o = TT_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o) sv[tid] += sv[tid + o];
        __syncthreads();
    }
    const double r = sv[0];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(TT_THREADS) tt_measure_kernel(const T *__restrict__ syn, const T *__restrict__ obs,
                                                               int n_t, int64_t n_rx, double dt, int M,
                                                               double *__restrict__ tau, T *__restrict__ ubar) {
    extern __shared__ double2 sh[];
    double2 *ss = sh, *sd = sh + 3 * n_t;                        // [j][c]
    double *C = reinterpret_cast<double *>(sd + 3 * n_t);        // [2M + 1]
    __shared__ double sv[TT_THREADS];
    __shared__ int sm[TT_THREADS];
    const int64_t r = blockIdx.x;
    const int tid = threadIdx.x;
    for (int q = tid; q < 3 * n_t; q += TT_THREADS) {
        const int j = q / 3, c = q - 3 * j;
        const int64_t g = ((int64_t)j * n_rx + r) * 3 + c;
        ss[q] = to_d2(syn[g]);
        sd[q] = to_d2(obs[g]);
    }
    __syncthreads();
    double best = -DBL_MAX;
    int bl = INT_MAX;
    for (int m = -M + tid; m <= M; m += TT_THREADS) {
        const int j0 = m < 0 ? -m : 0, j1 = m > 0 ? n_t - m : n_t;
        double acc = 0.0;
        for (int j = j0; j < j1; j++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const double2 a = ss[3 * j + c], b = sd[3 * (j + m) + c];
                acc = fma(a.x, b.x, fma(a.y, b.y, acc));
            }
        C[m + M] = acc;
        if (acc > best) {   // lags ascend per thread: the first maximum keeps the smallest lag
            best = acc;
            bl = m;
        }
    }
    argmax_block(best, bl, sv, sm);   // also orders the C[] stores before the reads below
    double t = (double)bl;
    if (bl > -M && bl < M) {
        const double a = C[bl + M - 1], b = C[bl + M], c = C[bl + M + 1];
        const double den = a - 2.0 * b + c;
        if (den < 0.0) t += (a - c) / (2.0 * den);
    }
    t *= dt;
    // N = (1/dt) sum_{j=-1}^{n_t-1} |s[j+1] - s[j]|^2 with s[-1] = s[n_t] = 0
    double part = 0.0;
    for (int q = tid; q < 3 * (n_t + 1); q += TT_THREADS) {
        const int j = q / 3 - 1, c = q - 3 * (q / 3);
        const double2 hi = j + 1 < n_t ? ss[3 * (j + 1) + c] : make_double2(0.0, 0.0);
        const double2 lo = j >= 0 ? ss[3 * j + c] : make_double2(0.0, 0.0);
        const double dx = hi.x - lo.x, dy = hi.y - lo.y;
        part = fma(dx, dx, fma(dy, dy, part));
    }
    const double N = sum_block(part, sv) / dt;
    if (tid == 0) tau[r] = t;
    if (ubar) {
        const double g = N > 0.0 ? t * dt / N : 0.0;
        const double h = g / (2.0 * dt);
        for (int q = tid; q < 3 * n_t; q += TT_THREADS) {
            const int j = q / 3, c = q - 3 * j;
            const double2 nx = j + 1 < n_t ? ss[q + 3] : make_double2(0.0, 0.0);
            const double2 pv = j > 0 ? ss[q - 3] : make_double2(0.0, 0.0);
            put(ubar + ((int64_t)j * n_rx + r) * 3 + c, h * (nx.x - pv.x), h * (nx.y - pv.y));
        }
    }
}

// misfit = 1/2 sum_r tau_r^2, one block, fixed order
__global__ void __launch_bounds__(TT_THREADS) tt_misfit_kernel(const double *__restrict__ tau, int64_t n_rx,
                                                              double *__restrict__ misfit) {
    __shared__ double sv[TT_THREADS];
    double part = 0.0;
    for (int64_t r = threadIdx.x; r < n_rx; r += TT_THREADS) part = fma(tau[r], tau[r], part);
    const double s = sum_block(part, sv);
    if (threadIdx.x == 0) *misfit = 0.5 * s;
}

template <typename T>
fga_status launch(const void *syn, const void *obs, int n_t, int64_t n_rx, double dt, int M, double *tau, void *ubar,
                  size_t smem, cudaStream_t s) {
    if (n_rx > 0) {
        auto kern = tt_measure_kernel<T>;
        if (smem > 48 * 1024) FGA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps(P_MISFIT, s);
        kern<<<(unsigned)n_rx, TT_THREADS, smem, s>>>(static_cast<const T *>(syn), static_cast<const T *>(obs), n_t,
                                                      n_rx, dt, M, tau, static_cast<T *>(ubar));
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" fga_status fga_traveltime_adjoint(const void *syn, const void *obs, int precision, int64_t n_times,
                                             int64_t n_rx, double dt, int max_lag, double *tau, void *ubar,
                                             double *misfit, fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(precision == FGA_PREC_FP32 || precision == FGA_PREC_FP64, "fga_traveltime_adjoint: bad precision");
    FGA_CHECK(n_times >= 1 && n_rx >= 0, "fga_traveltime_adjoint: n_times >= 1 and n_rx >= 0");
    FGA_CHECK(std::isfinite(dt) && dt > 0.0, "fga_traveltime_adjoint: dt must be finite and > 0");
    FGA_CHECK(max_lag >= 0 && (int64_t)max_lag < n_times, "fga_traveltime_adjoint: 0 <= max_lag < n_times");
    FGA_CHECK(n_rx == 0 || (syn && obs && tau), "fga_traveltime_adjoint: syn, obs and tau are required");
    FGA_CHECK(n_rx <= INT_MAX, "fga_traveltime_adjoint: too many receivers");
    const size_t smem = sizeof(double2) * 6 * (size_t)n_times + sizeof(double) * (2 * (size_t)max_lag + 1);
    FGA_CHECK(smem <= 200 * 1024, "fga_traveltime_adjoint: records too long for the shared-memory stage "
                                  "(96 n_times + 16 max_lag bytes must stay within 200 KiB)");
    const int n_t = (int)n_times, M = max_lag;
    if (precision == FGA_PREC_FP32)
        FGA_TRY(launch<float2>(syn, obs, n_t, n_rx, dt, M, tau, ubar, smem, s));
    else
        FGA_TRY(launch<double2>(syn, obs, n_t, n_rx, dt, M, tau, ubar, smem, s));
    if (misfit) {
        ProfScope ps(P_MISFIT, s);
        if (n_rx > 0)
            tt_misfit_kernel<<<1, TT_THREADS, 0, s>>>(tau, n_rx, misfit);
        else
            FGA_CUDA(cudaMemsetAsync(misfit, 0, sizeof(double), s));
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}
