// Complex GEMMs of the wave-packet transform (A1) on the 5th-generation tensor cores, FP16 split
// precision with FP32 accumulation:
//
//   C[z][m][n] = scale * sum_k A[z][m][k] B[n][k]        (complex; |B| <= 1: the per-axis kernels)
//
// Complex -> real: with A' = [Re A | Im A] (M x 2K) and the two K-halves of B'
//   B'_re = [Re B ; Im B]   (rows n: Re C, rows n_c + n: Im C),   B'_im = [-Im B ; Re B],
// Re/Im C = A'_re B'_re^T + A'_im B'_im^T, one real GEMM of width 2 n_c per N tile.
// FP16 split: x = hi + lo with hi = fp16(x), lo = fp16(x - hi); each real product is
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), three tcgen05.mma per K step, all
// accumulating into one FP32 tile in tensor memory.  Operands are scaled by exact powers of two so that
// hi and lo stay in the FP16 normal range (A by a bound on |A| read from device memory, B by 2^14).
//
// One CTA = one 128-row M tile x one N tile (2 n_c <= 256 real columns), 128 threads:
//   all threads stage a K block of A' and B' (hi and lo) into shared memory in the canonical
//   no-swizzle K-major layout (8x8 core matrices of 128 contiguous bytes), one elected thread issues
//   the MMAs and commits them to an mbarrier; after the last block the four warps read their 32 TMEM
//   lanes (rows) and write C.  Every wait is bounded: a wait that runs out sets *err, waits once more
//   (bounded) for the outstanding commit, and then frees its tensor memory without writing C.
#include <cuda_fp16.h>

#include <cmath>

#include "fga_beam.cuh"
#include "tcgen05.cuh"

namespace fga {
namespace {

constexpr int TC_M = 128;      // rows per tile (TMEM lanes)
constexpr int TC_KB = tc::KB;  // complex K per staged block (real K per half = 32: two MMA K steps)
constexpr int TC_NMAX = 256;   // real columns per tile (TMEM columns allocated)
constexpr uint32_t TC_TMEM_COLS = 256;

// shared memory of one K block: [A'_re hi, A'_re lo, A'_im hi, A'_im lo] (128 x 32 fp16 each) and
// [B'_re hi, B'_re lo, B'_im hi, B'_im lo] (NR x 32 fp16 each, NR <= 256)
constexpr int TC_A_BYTES = TC_M * TC_KB * 2;           // 8 KB
constexpr int TC_B_BYTES = TC_NMAX * TC_KB * 2;        // 16 KB
constexpr int TC_SMEM = 4 * TC_A_BYTES + 4 * TC_B_BYTES + 1024;  // 96 KB + barrier/bookkeeping

// grid: (M tiles, N tiles, Z); block 128; dynamic shared memory TC_SMEM
template <typename TA>
__global__ void __launch_bounds__(128, 1) tc_cgemm_kernel(const TA *__restrict__ A, int64_t sAz, int64_t sAm,
                                                         int64_t sAk, const float2 *__restrict__ B, int64_t sBn,
                                                         int64_t sBk, float2 *__restrict__ C, int64_t sCz,
                                                         int64_t sCm, int64_t sCn, int64_t M, int N, int K,
                                                         int nc_tile, float scale, const float *__restrict__ amax,
                                                         float amax_factor, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                       // 4 x TC_A_BYTES
    unsigned char *sB = smem + 4 * TC_A_BYTES;      // 4 x TC_B_BYTES
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 4 * TC_A_BYTES + 4 * TC_B_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * TC_M;
    const int n0 = blockIdx.y * nc_tile;
    const int nc = min(nc_tile, N - n0);   // complex columns of this tile
    const int NR = 2 * nc_tile;            // real MMA width (fixed per launch; unused rows are zero)

    // operand scales: A so that |A| * sa <= 2^14, B (|B| <= 1) by 2^14
    float sa = 1.0f;
    {
        const float bound = amax ? (*amax) * amax_factor : 1.0f;
        if (bound > 0.0f && isfinite(bound)) {
            int e;
            frexpf(bound, &e);          // bound < 2^e
            sa = ldexpf(1.0f, 14 - e);
        }
    }
    const float sb = 16384.0f;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::instr_desc(NR, TC_M);
    const TA *Az = A + (int64_t)z * sAz;
    const bool rowfast = sAm <= sAk;   // consecutive threads take consecutive rows when rows are closer
    uint32_t parity = 0;
    bool ok = true;
    const int nkb = (K + TC_KB - 1) / TC_KB;
    for (int kb = 0; kb < nkb && ok; kb++) {
        const int k0 = kb * TC_KB;
        // ---- stage A' (128 rows x 32 complex k) ----
        for (int e = tid; e < TC_M * TC_KB; e += 128) {
            const int row = rowfast ? (e % TC_M) : (e / TC_KB);
            const int kk = rowfast ? (e / TC_M) : (e % TC_KB);
            const int64_t gm = m0 + row;
            const int gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (gm < M && gk < K) v = tc::ld_c<TA>(Az + gm * sAm + (int64_t)gk * sAk);
            const uint32_t off = tc::kmaj_off(row, kk);
            tc::split_store(sA + 0 * TC_A_BYTES, sA + 1 * TC_A_BYTES, off, v.x * sa);
            tc::split_store(sA + 2 * TC_A_BYTES, sA + 3 * TC_A_BYTES, off, v.y * sa);
        }
        // ---- stage B'_re = [Re B ; Im B], B'_im = [-Im B ; Re B] (NR rows x 32 k) ----
        for (int e = tid; e < nc_tile * TC_KB; e += 128) {
            const int j = e / TC_KB, kk = e % TC_KB;
            const int gn = n0 + j, gk = k0 + kk;
            float2 v = make_float2(0.f, 0.f);
            if (j < nc && gk < K) v = B[(int64_t)gn * sBn + (int64_t)gk * sBk];
            const float br = v.x * sb, bi = v.y * sb;
            const uint32_t o_top = tc::kmaj_off(j, kk), o_bot = tc::kmaj_off(nc_tile + j, kk);
            tc::split_store(sB + 0 * TC_B_BYTES, sB + 1 * TC_B_BYTES, o_top, br);
            tc::split_store(sB + 0 * TC_B_BYTES, sB + 1 * TC_B_BYTES, o_bot, bi);
            tc::split_store(sB + 2 * TC_B_BYTES, sB + 3 * TC_B_BYTES, o_top, -bi);
            tc::split_store(sB + 2 * TC_B_BYTES, sB + 3 * TC_B_BYTES, o_bot, br);
        }
        // make the generic-proxy stores visible to the tensor cores, then issue
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            // per K half (re, im): two K steps of 16; per step hi*hi, hi*lo, lo*hi
            for (int half = 0; half < 2; half++) {
                const uint32_t a_hi = tc::smem_u32(sA + (2 * half) * TC_A_BYTES), a_lo = tc::smem_u32(sA + (2 * half + 1) * TC_A_BYTES);
                const uint32_t b_hi = tc::smem_u32(sB + (2 * half) * TC_B_BYTES), b_lo = tc::smem_u32(sB + (2 * half + 1) * TC_B_BYTES);
                for (int ks = 0; ks < TC_KB / 16; ks++) {
                    const uint32_t koff = ks * 2 * 128;   // two core matrices along K
                    const uint64_t dah = tc::smem_desc(a_hi + koff), dal = tc::smem_desc(a_lo + koff);
                    const uint64_t dbh = tc::smem_desc(b_hi + koff), dbl = tc::smem_desc(b_lo + koff);
                    const uint32_t acc0 = (kb > 0 || half > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(dah), "l"(dbh), "r"(idesc), "r"(acc0)
                        : "memory");
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(dah), "l"(dbl), "r"(idesc), "r"(1u)
                        : "memory");
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(dal), "l"(dbh), "r"(idesc), "r"(1u)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc::smem_u32(bar))
                         : "memory");
        }
        // the MMAs read shared memory until the commit arrives: wait before restaging
        bool arrived = true;
        if (tid == 0) arrived = tc::mbar_wait(tc::smem_u32(bar), parity);   // one poller
        ok = __syncthreads_and(arrived ? 1 : 0) != 0;   // uniform across the CTA
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) parity ^= 1u;
    }
    // give-up: report, and let the outstanding commit (phase `parity`) land before freeing its columns
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        tc::mbar_drain(tc::smem_u32(bar), parity);
    }
    if (ok) {
        // ---- epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31 ----
        const int row = warp * 32 + lane;
        const int64_t gm = m0 + row;
        const float inv = scale / (sa * sb);
        float2 *Cz = C + (int64_t)z * sCz;
        for (int c0 = 0; c0 < nc_tile; c0 += 8) {
            uint32_t re[8], im[8];
            const uint32_t tre = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            const uint32_t tim = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(nc_tile + c0);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(re[0]), "=r"(re[1]), "=r"(re[2]), "=r"(re[3]), "=r"(re[4]), "=r"(re[5]), "=r"(re[6]),
                           "=r"(re[7])
                         : "r"(tre)
                         : "memory");
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(im[0]), "=r"(im[1]), "=r"(im[2]), "=r"(im[3]), "=r"(im[4]), "=r"(im[5]), "=r"(im[6]),
                           "=r"(im[7])
                         : "r"(tim)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (gm < M) {
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int j = c0 + q;
                    if (j < nc)
                        Cz[gm * sCm + (int64_t)(n0 + j) * sCn] =
                            make_float2(__uint_as_float(re[q]) * inv, __uint_as_float(im[q]) * inv);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

__global__ void absmax_kernel(const double2 *__restrict__ x, int64_t n, float *__restrict__ out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        m = fmaxf(m, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));  // m >= 0
}

}  // namespace

// |x|_max of complex double data into *out (DEVICE float, zeroed here)
fga_status tc_absmax(const double2 *x, int64_t n, float *out, cudaStream_t s) {
    FGA_CUDA(cudaMemsetAsync(out, 0, sizeof(float), s));
    const int blocks = (int)std::min<int64_t>(152 * 8, (n + 255) / 256 + 1);
    absmax_kernel<<<blocks, 256, 0, s>>>(x, n, out);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

template <typename TA>
fga_status tc_cgemm(const TA *A, int64_t sAz, int64_t sAm, int64_t sAk, const float2 *B, int64_t sBn, int64_t sBk,
                    float2 *C, int64_t sCz, int64_t sCm, int64_t sCn, int Z, int64_t M, int N, int K, float scale,
                    const float *amax, float amax_factor, int *err, cudaStream_t s) {
    const int ntile = (N + 127) / 128;                      // 2 n_c <= 256 real columns per tile
    const int nc_tile = ((N + ntile - 1) / ntile + 7) / 8 * 8;   // multiple of 8 (MMA N multiple of 16)
    FGA_CUDA(cudaFuncSetAttribute(tc_cgemm_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    dim3 grid((unsigned)((M + TC_M - 1) / TC_M), (unsigned)ntile, (unsigned)Z);
    ProfScope ps(P_DECOMP, s);
    tc_cgemm_kernel<TA><<<grid, 128, TC_SMEM, s>>>(A, sAz, sAm, sAk, B, sBn, sBk, C, sCz, sCm, sCn, M, N, K, nc_tile,
                                                   scale, amax, amax_factor, err);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

template fga_status tc_cgemm<double2>(const double2 *, int64_t, int64_t, int64_t, const float2 *, int64_t, int64_t,
                                      float2 *, int64_t, int64_t, int64_t, int, int64_t, int, int, float, const float *,
                                      float, int *, cudaStream_t);
template fga_status tc_cgemm<float2>(const float2 *, int64_t, int64_t, int64_t, const float2 *, int64_t, int64_t,
                                     float2 *, int64_t, int64_t, int64_t, int, int64_t, int, int, float, const float *,
                                     float, int *, cudaStream_t);

}  // namespace fga
