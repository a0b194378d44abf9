// fga_reconstruct_noalloc: the Gaussian sum at points (the same result as fga_reconstruct) for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc/cudaFree are unavailable or unsafe -- for example
// a host callback or a real-time loop that must not block on the allocator's implicit device
// synchronisation, a process whose memory is carved up in advance by an outside pool manager, or
// a plug-in that is handed device buffers but no allocation rights.  fga_reconstruct grows
// library-owned scratch on demand (records, sort buffers, partial sums), so it may call cudaMalloc;
// this variant never does.
//
// How: its only scratch is the file-scope device array g_noalloc_scratch below (12 MiB; every GPU
// that loads the library keeps it until the process exits).  It holds the per-chunk partial sums of
// a brute-force gather: every point is tested against every beam (no cell binning, which would need
// scratch proportional to the beam count).  The first call on a device looks up the array's device
// address with cudaGetSymbolAddress (host code may not use the symbol itself: on the host it is only
// a stand-in).  With CUDA's lazy module loading that lookup may also load this file's module on the
// device and place the array there -- a one-time cost that can synchronise the device -- so a caller
// that must never stall makes one warm-up call with n = 0 first, which does only this set-up.  Every
// call overwrites all the partial sums it later reads, so nothing has to start at zero; calls that
// overlap on the GPU (two streams at once) share the array and race.
#include <cmath>
#include <mutex>

#include "fga_beam.cuh"
#include "gather.cuh"

namespace fga {
namespace {

constexpr int NA_CHUNKS = 64;          // beam chunks per call (partial sums per point)
constexpr int NA_MAX_POINTS = 4096;    // largest point count one call accepts
constexpr size_t NA_SCRATCH_BYTES = (size_t)NA_CHUNKS * NA_MAX_POINTS * 6 * sizeof(double);  // 12 MiB
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

std::mutex g_na_mutex;
void *g_na_ptr[NA_MAX_DEVICES] = {};

// device address of the scratch array on the current device (looked up once per device)
fga_status scratch_ptr(void **out) {
    int dev = -1;
    FGA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        set_error("fga_reconstruct_noalloc: device ordinal out of range");
        return FGA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return FGA_OK;
}

// partial[chunk][point][6]: the sum over the chunk's beams for each point of a 32-point tile.
// Lanes own points; the four warps split the chunk; the record of a beam is formed on the fly from
// its state (the same record the library's own gather uses).
template <typename R, int WAVE>
__global__ void __launch_bounds__(128) noalloc_gather_kernel(const R *__restrict__ st, const int32_t *__restrict__ flags,
                                                            int64_t cap, int64_t beg, int64_t nbeams, R w,
                                                            const double *__restrict__ x, int64_t npts, R k, R rw2,
                                                            int chunk0, R *__restrict__ partial, int accumulate) {
    __shared__ R red[4][32][6];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.y * 32 + lane;
    R x0 = R(1e30), x1 = R(1e30), x2 = R(1e30);
    if (p < npts) {
        x0 = (R)x[3 * p];
        x1 = (R)x[3 * p + 1];
        x2 = (R)x[3 * p + 2];
    }
    const int chunk = blockIdx.x;
    const int64_t c0 = beg + (nbeams * chunk) / NA_CHUNKS, c1 = beg + (nbeams * (chunk + 1)) / NA_CHUNKS;
    const int64_t len = c1 - c0;
    const int64_t b0 = c0 + (len * warp) / 4, b1 = c0 + (len * (warp + 1)) / 4;
    R acc[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const R hk = R(-0.5) * k;
    for (int64_t b = b0; b < b1; b++) {
        R y[NF];
#pragma unroll
        for (int f = 0; f < 6; f++) y[f] = st[(int64_t)f * cap + b];
#pragma unroll
        for (int f = F_A0; f < NF; f++) y[f] = st[(int64_t)f * cap + b];
#pragma unroll
        for (int d = 0; d < 3; d++) y[F_Q + d] -= st[(int64_t)(F_QC + d) * cap + b];   // compensated Q
        R r[REC];
        beam_record<R, WAVE>((flags[b] & FL_REF_E1) != 0, y, y, y, y, R(0), R(0), w, r);
        const R d0 = x0 - r[0], d1 = x1 - r[1], d2 = x2 - r[2];
        const R r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 <= rw2) {
            const R ph = k * (r[3] * d0 + r[4] * d1 + r[5] * d2);
            R er, ei;
            gauss_phase_exp<R>(ph, hk * r2, &er, &ei);
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const R ar = r[6 + 2 * d], ai = r[7 + 2 * d];
                acc[2 * d] += ar * er - ai * ei;
                acc[2 * d + 1] += ar * ei + ai * er;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 6; j++) red[warp][lane][j] = acc[j];
    __syncthreads();
    if (warp == 0 && p < npts) {
        R *dst = partial + ((int64_t)chunk * NA_MAX_POINTS + p) * 6;
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const R v = (red[0][lane][j] + red[1][lane][j]) + (red[2][lane][j] + red[3][lane][j]);
            dst[j] = accumulate ? dst[j] + v : v;  // classes after the first add to the same slot
        }
    }
}

template <typename R>
__global__ void noalloc_reduce_kernel(const R *__restrict__ partial, int64_t npts, R *__restrict__ u) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int c = 0; c < NA_CHUNKS; c++)
#pragma unroll
        for (int j = 0; j < 6; j++) acc[j] += (double)partial[((int64_t)c * NA_MAX_POINTS + p) * 6 + j];
#pragma unroll
    for (int j = 0; j < 6; j++) u[p * 6 + j] = (R)acc[j];
}

template <typename R>
fga_status run_noalloc(const fga_beams *b, const double *x, int64_t n, R rw, void *u_out, void *scratch,
                       cudaStream_t s) {
    R *partial = static_cast<R *>(scratch);
    const dim3 grid(NA_CHUNKS, (unsigned)((n + 31) / 32));
    int first = 1;
    for (int cls = 0; cls < 4; cls++) {
        const int64_t nc = b->n_cls[cls];
        if (nc == 0) continue;
        const int acc = first ? 0 : 1;
        if (cls < 2)
            noalloc_gather_kernel<R, 0><<<grid, 128, 0, s>>>(b->state.as<R>(), b->flags.as<int32_t>(), b->cap,
                                                             b->off_cls[cls], nc, (R)b->w, x, n, (R)b->k, rw * rw, 0,
                                                             partial, acc);
        else
            noalloc_gather_kernel<R, 1><<<grid, 128, 0, s>>>(b->state.as<R>(), b->flags.as<int32_t>(), b->cap,
                                                             b->off_cls[cls], nc, (R)b->w, x, n, (R)b->k, rw * rw, 0,
                                                             partial, acc);
        first = 0;
    }
    FGA_CUDA(cudaGetLastError());
    if (first) {  // no beams at all: the sum is zero
        FGA_CUDA(cudaMemsetAsync(u_out, 0, sizeof(R) * 6 * (size_t)n, s));
        return FGA_OK;
    }
    noalloc_reduce_kernel<R><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(partial, n, static_cast<R *>(u_out));
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" fga_status fga_reconstruct_noalloc(const fga_beams *b, const double *x, int64_t n, double rw, void *u_out,
                                              fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(b, "fga_reconstruct_noalloc: NULL beams");
    FGA_CHECK(!b->tilted, "fga_reconstruct_noalloc: beams of tilted layers are not supported");
    if (b->layered) {
        set_error("fga_reconstruct_noalloc: beams of a layered medium are not supported");
        return FGA_ERR_UNSUPPORTED;
    }
    FGA_CHECK(n >= 0, "fga_reconstruct_noalloc: n < 0");
    void *scratch = nullptr;
    FGA_TRY(scratch_ptr(&scratch));   // n = 0: only this one-time set-up (a warm-up call)
    if (n == 0) return FGA_OK;
    FGA_CHECK(n <= NA_MAX_POINTS,
              "fga_reconstruct_noalloc: more than 4096 points in one call (its fixed scratch holds the partial sums "
              "of at most 4096 points); split the points or use fga_reconstruct");
    FGA_CHECK(x && u_out, "fga_reconstruct_noalloc: NULL points or output");
    if (!(rw > 0)) rw = 6.0 / std::sqrt(b->k);
    if (b->precision == FGA_PREC_FP64) return run_noalloc<double>(b, x, n, rw, u_out, scratch, s);
    return run_noalloc<float>(b, x, n, (float)rw, u_out, scratch, s);
}
