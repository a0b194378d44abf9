// A6 on single-plane lattices (receiver arrays: n0 x n1 points at one x3), FP32 path, on the
// tensor cores with warp-specialised producers.
//
// On a tile of T0 x T1 points of the plane, with E_d the per-axis Gaussian factors of Eq. FGA,
//
//   U[(j,c)][i] = sum_b  W_bc E1_b(x_j) E0_b(x_i),      W_bc = A_bc E2_b(x_2)
//
// is a complex matrix product over the beams b (the contraction index): rows (j, c) -> TMEM lanes
// r = 32 h + 3 t + c with j = h J + t (J = ceil(T1/2), h in {0, 1}), columns i -> Re/Im of the
// accumulator (C' = A_re B'_re^T + A_im B'_im^T with B'_re = [Re E0; Im E0], B'_im = [-Im E0; Re E0]).
// Both operands are FP16 hi/lo splits of the FP32 values (hi*hi + hi*lo + lo*hi, FP32 accumulation),
// as in the other tensor-core kernels of the library.
//
// One persistent CTA per SM: eight producer warps and one MMA warp.
//  - Each producer warp filters its share of an item's candidate records (the beams within the window
//    radius of the tile's box) into a queue and turns every 32 kept beams into one operand block: lane
//    (h, p) takes beams 2p and 2p+1, forms E0 by a stride-2 recurrence on its parity (the other parity
//    comes from lane p + 16h' by a shuffle), E1 by recurrence on its half of the rows, W, and writes
//    32-bit pairs of FP16 values straight into the K-major operand layout.  The layout is padded
//    (leading byte offset 144, row-group stride chosen per tile) so that these stores are free of bank
//    conflicts.
//  - Blocks are numbered in the order they are claimed and go through a ring of shared-memory stages;
//    per stage a "full" mbarrier (producer -> MMA) and an "empty" one (tcgen05.commit -> producers).
//  - The MMA warp's elected thread issues 12 tcgen05.mma (two K steps x re/im x three split products)
//    per block into an M = 128 x N = 2 n_c accumulator; rows 64..127 of the A descriptor read the
//    neighbouring buffer and their accumulator lanes are never read.
//  - At the end of an item an END block (no data) closes the sequence; after the last commit the
//    accumulator rows go to the plan's per-item partial sums, reduced as for the other lattice kernels.
// Every wait is bounded: a wait that runs out sets the CTA's abort flag and the call's error word; an
// aborting CTA keeps its barrier schedule, issues no further MMA, waits (bounded) for its outstanding
// commit and frees its tensor memory.
#include <algorithm>
#include <cmath>

#include "fga_beam.cuh"
#include "gather.cuh"
#include "tcgen05.cuh"

namespace fga {

// in-window pairs counted by the counting instantiation (profiling)
static __device__ unsigned long long g_plane_pairs;

int64_t read_plane_pair_counter(bool reset) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_plane_pairs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_plane_pairs, &z, sizeof z);
    }
    return (int64_t)v;
}

namespace {

constexpr int PL_PROD = 8;                     // producer warps
constexpr int PL_THREADS = (PL_PROD + 1) * 32; // + the MMA warp
constexpr int PL_KB = 32;                      // beams per block
constexpr int PL_STAGES = 6;                   // most stages (fewer when a stage is large)
constexpr int PL_LBO = 144;                    // bytes between K-adjacent core matrices
constexpr int PL_SBO_A = 592;                  // bytes between row-adjacent core matrices of A
constexpr int PL_A_COPY = 8 * PL_SBO_A;        // one A copy: 64 rows (8 row groups)
constexpr int PL_QUEUE = 64;                   // kept-beam queue per producer warp
constexpr int PL_T0_MAX = 32, PL_T1_MAX = 20;

struct PlaneArgs {
    const float *rec;        // records [n_rec][12]: Q, P, weighted polarised amplitude (3 complex)
    const int4 *items;       // (tile, first record, end record, 0)
    int nitems;
    int n0, n1;              // lattice extents (n2 = 1)
    int T0, T1, nt1;         // tile shape and tiles along axis 1
    int nc;                  // complex accumulator columns (T0 rounded up to 8)
    int sbo_b;               // row-group stride of the B copies
    int b_copy, stage_bytes, nst;
    float x0, h0, x1, h1, x2;  // uniform axes 0 and 1, the plane's x3
    float k, rw2;
    const float *amax;       // bound of |A| over the records
    float *partial;          // [item][T0*T1][6]
    int *err;
    uint32_t tcols;
};

__device__ __forceinline__ uint32_t koff(int row, int kk, int sbo) {
    return (uint32_t)((row >> 3) * sbo + (kk >> 3) * PL_LBO + (row & 7) * 16 + (kk & 7) * 2);
}

// FP16 hi/lo split of the pair (a, b), packed as two f16x2 words
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 hh = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&hh);
    lo = *reinterpret_cast<const uint32_t *>(&ll);
}

__device__ __forceinline__ void sts32(unsigned char *base, uint32_t off, uint32_t v) {
    *reinterpret_cast<uint32_t *>(base + off) = v;
}

// bounded wait (2^22 polls; the stages turn over in microseconds), which also gives up once any CTA of
// the launch has reported a timeout in the call's error word
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, const int *gerr) {
    for (int it = 0; it < (1 << 22); it++) {
        uint32_t ready;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ready)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ready) return true;
        if ((it & 1023) == 1023 && *reinterpret_cast<const volatile int *>(gerr) != 0) return false;
    }
    return false;
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// A stage's empty barrier is waited on by parity, which only tells its newest phase from the one
// before.  Blocks are claimed by several producers, so the producer of block n first waits until the
// MMA thread has taken block n - nst (the stage's previous use): then the stage's use before that has
// completed, and the parity wait below refers to the right phase.
__device__ __forceinline__ bool wait_taken(const int *taken, int need, const int *gerr) {
    for (int it = 0; it < (1 << 22); it++) {
        if (*reinterpret_cast<const volatile int *>(taken) >= need) return true;
        if ((it & 1023) == 1023 && *reinterpret_cast<const volatile int *>(gerr) != 0) return false;
    }
    return false;
}

// first wait of a launch that gave up: the error word plus where (1 producer stage wait, 2 END stage
// wait, 3 MMA wait for a block, 4 wait for the item's last commit), the block, its stage and parity,
// the blocks claimed and the CTA (words 2..7 of the call's status words)
__device__ __forceinline__ void report_timeout(int *err, int site, int n, int s, int parity, int claimed, int consumed) {
    atomicExch(err, 1);
    if (atomicCAS(err + 2, 0, site) == 0) {
        err[3] = n;
        err[4] = s;
        err[5] = parity;
        err[6] = claimed;
        err[7] = blockIdx.x;
        err[8] = consumed;
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <bool COUNT>
__global__ void __launch_bounds__(PL_THREADS, 1) plane_tc_kernel(PlaneArgs P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *stages = smem;
    unsigned char *tail = smem + P.nst * P.stage_bytes + PL_A_COPY;   // A rows 64..127 may read past the ring
    uint64_t *full = reinterpret_cast<uint64_t *>(tail);
    uint64_t *empty = full + PL_STAGES;
    uint64_t *done = empty + PL_STAGES;
    int *hdr = reinterpret_cast<int *>(done + 1);          // per stage: beams in the block, -1 = END
    int *misc = hdr + PL_STAGES;                           // 0 blocks claimed, 1 abort, 2 item had MMAs, 3 blocks taken by the MMA thread
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(misc + 4);
    int *queues = reinterpret_cast<int *>(misc + 8);       // [PL_PROD][PL_QUEUE]

    if (warp == PL_PROD) tc::alloc(tc::smem_u32(tmem_slot), P.tcols);
    if (tid == 0) {
        for (int s = 0; s < P.nst; s++) {
            tc::mbar_init(tc::smem_u32(full + s));
            tc::mbar_init(tc::smem_u32(empty + s));
        }
        tc::mbar_init(tc::smem_u32(done));
        misc[0] = 0;
        misc[1] = 0;
        misc[3] = 0;
    }
    float sa = 1.0f;
    {
        const float bound = *P.amax;
        if (bound > 0.0f && isfinite(bound)) {
            int e;
            frexpf(bound, &e);
            sa = ldexpf(1.0f, 14 - e);
        }
    }
    const float sb = 16384.0f;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int *abort_flag = misc + 1;

    const int J = (P.T1 + 1) >> 1;           // j values per row half
    const int NR = 2 * P.nc;
    const float hk = -0.5f * P.k;
    uint32_t done_par = 0;
    int mma_n = 0;                           // next block the MMA thread consumes (never reset)

    for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
        const int4 it = P.items[item];
        const int t = it.x, tt0 = t / P.nt1, tt1 = t % P.nt1;
        const int i0 = tt0 * P.T0, j0 = tt1 * P.T1;
        const int e0 = min(P.T0, P.n0 - i0), e1 = min(P.T1, P.n1 - j0);
        // the tile's box (window test of the candidates)
        const float blo0 = P.x0 + P.h0 * i0, bhi0 = P.x0 + P.h0 * (i0 + e0 - 1);
        const float blo1 = P.x1 + P.h1 * j0, bhi1 = P.x1 + P.h1 * (j0 + e1 - 1);
        if (warp < PL_PROD) {
            // ------------------------------------------------ producers ----------------------------
            int *q = queues + warp * PL_QUEUE;
            int qh = 0, qt = 0;
            const int h = lane >> 4, p = lane & 15;
            unsigned long long pairs = 0;
            auto produce = [&](int nvalid) {
                // claim the next block number and its stage
                int n = 0;
                if (lane == 0) n = atomicAdd(misc + 0, 1);
                n = __shfl_sync(0xffffffffu, n, 0);
                const int s = n % P.nst, use = n / P.nst;
                bool ok = *abort_flag == 0;
                if (use > 0 && ok) {
                    bool w = true;
                    if (lane == 0)
                        w = wait_taken(misc + 3, n - P.nst + 1, P.err) &&
                            bar_wait(tc::smem_u32(empty + s), (uint32_t)((use - 1) & 1), P.err);
                    w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
                    if (!w) {
                        if (lane == 0) {
                            *abort_flag = 1;
                            report_timeout(P.err, 1, n, s, (use - 1) & 1, misc[0], misc[3]);
                        }
                        ok = false;
                    }
                }
                unsigned char *st = stages + s * P.stage_bytes;
                unsigned char *Are = st, *Are_lo = st + PL_A_COPY, *Aim = st + 2 * PL_A_COPY,
                              *Aim_lo = st + 3 * PL_A_COPY;
                unsigned char *Bre = st + 4 * PL_A_COPY, *Bre_lo = Bre + P.b_copy, *Bim = Bre + 2 * P.b_copy,
                              *Bim_lo = Bre + 3 * P.b_copy;
                if (ok) {
                    // the two beams of this lane
                    float2 W[2][3];
                    float2 f1[2], q1[2], f0[2], q0[2];
                    float g1 = 1.f, g0 = 1.f;
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        const int slot = 2 * p + u;
                        float r[REC];
                        if (slot < nvalid) {
                            const float4 *src = reinterpret_cast<const float4 *>(P.rec + (int64_t)q[(qh + slot) & (PL_QUEUE - 1)] * REC);
                            const float4 a = src[0], b = src[1], c = src[2];
                            r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
                            r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
                            r[8] = c.x; r[9] = c.y; r[10] = c.z; r[11] = c.w;
                        } else {
#pragma unroll
                            for (int f = 0; f < REC; f++) r[f] = 0.f;
                        }
                        // W_c = A_c E2 (scaled for the A operand); zero for padding beams
                        const float dz = P.x2 - r[2];
                        float er, ei;
                        gauss_phase_exp<float>(P.k * r[5] * dz, hk * dz * dz, &er, &ei);
                        const float scl = slot < nvalid ? sa : 0.f;
#pragma unroll
                        for (int c = 0; c < 3; c++)
                            W[u][c] = make_float2(scl * (r[6 + 2 * c] * er - r[7 + 2 * c] * ei),
                                                  scl * (r[6 + 2 * c] * ei + r[7 + 2 * c] * er));
                        // E1 at x_j, j = j0 + h J (start of this half), and its ratio for a step h1
                        {
                            const float d = P.x1 + P.h1 * (float)(j0 + h * J) - r[1];
                            float a0r, a0i, rr, ri;
                            gauss_phase_exp<float>(P.k * r[4] * d, hk * d * d, &a0r, &a0i);
                            gauss_phase_exp<float>(P.k * r[4] * P.h1, -P.k * P.h1 * (d + 0.5f * P.h1), &rr, &ri);
                            f1[u] = make_float2(a0r, a0i);
                            q1[u] = make_float2(rr, ri);
                        }
                        // E0 at x_i, i = i0 + h (this lane's parity), and its ratio for a step 2 h0
                        {
                            const float d = P.x0 + P.h0 * (float)(i0 + h) - r[0];
                            const float s2 = 2.f * P.h0;
                            float a0r, a0i, rr, ri;
                            gauss_phase_exp<float>(P.k * r[3] * d, hk * d * d, &a0r, &a0i);
                            gauss_phase_exp<float>(P.k * r[3] * s2, -P.k * s2 * (d + 0.5f * s2), &rr, &ri);
                            const float valid = slot < nvalid ? sb : 0.f;
                            f0[u] = make_float2(valid * a0r, valid * a0i);
                            q0[u] = make_float2(rr, ri);
                        }
                        if (COUNT && slot < nvalid) {
                            // pairs of this beam inside the window, rows of this half
                            const float dz2 = (P.x2 - r[2]) * (P.x2 - r[2]);
                            for (int jj = h * J; jj < min(e1, (h + 1) * J); jj++) {
                                const float dy = P.x1 + P.h1 * (float)(j0 + jj) - r[1];
                                const float s2 = P.rw2 - dz2 - dy * dy;
                                if (s2 < 0.f) continue;
                                const float sq = sqrtf(s2);
                                if (P.h0 > 0.f) {
                                    const int lo = max(0, (int)ceilf((r[0] - sq - blo0) / P.h0));
                                    const int hi = min(e0 - 1, (int)floorf((r[0] + sq - blo0) / P.h0));
                                    if (hi >= lo) pairs += (unsigned long long)(hi - lo + 1);
                                } else if (fabsf(r[0] - blo0) <= sq) {
                                    pairs += 1ull;
                                }
                            }
                        }
                    }
                    g1 = __expf(-P.k * P.h1 * P.h1);
                    g0 = __expf(-4.f * P.k * P.h0 * P.h0);
                    // ---- A: rows r = 32 h + 3 t + c, j = h J + t ----
                    for (int tj = 0; tj < J; tj++) {
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const int row = 32 * h + 3 * tj + c;
                            const float2 v0 = cmul(W[0][c], f1[0]), v1 = cmul(W[1][c], f1[1]);
                            uint32_t rh, rl, ih, il;
                            split2(v0.x, v1.x, rh, rl);
                            split2(v0.y, v1.y, ih, il);
                            const uint32_t o = koff(row, 2 * p, PL_SBO_A);
                            sts32(Are, o, rh);
                            sts32(Are_lo, o, rl);
                            sts32(Aim, o, ih);
                            sts32(Aim_lo, o, il);
                        }
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            f1[u] = cmul(f1[u], q1[u]);
                            q1[u].x *= g1;
                            q1[u].y *= g1;
                        }
                    }
                    // ---- B: B're = [Re E0; Im E0], B'im = [-Im E0; Re E0]; half 0 stores the Re words,
                    // half 1 the Im words; each half forms E0 on its parity and gets the other one ----
                    for (int i2 = 0; i2 < P.T0; i2 += 2) {
                        float2 mine[2] = {f0[0], f0[1]}, other[2];
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            other[u].x = __shfl_xor_sync(0xffffffffu, mine[u].x, 16);
                            other[u].y = __shfl_xor_sync(0xffffffffu, mine[u].y, 16);
                        }
#pragma unroll
                        for (int par = 0; par < 2; par++) {
                            const int i = i2 + par;
                            if (i >= P.T0) break;
                            const float2 v0 = (par == h) ? mine[0] : other[0];
                            const float2 v1 = (par == h) ? mine[1] : other[1];
                            uint32_t wh, wl;
                            split2(h == 0 ? v0.x : v0.y, h == 0 ? v1.x : v1.y, wh, wl);
                            const uint32_t ra = koff(h == 0 ? i : P.nc + i, 2 * p, P.sbo_b);
                            const uint32_t rb = koff(h == 0 ? P.nc + i : i, 2 * p, P.sbo_b);
                            const uint32_t neg = h == 0 ? 0u : 0x80008000u;
                            sts32(Bre, ra, wh);
                            sts32(Bre_lo, ra, wl);
                            sts32(Bim, rb, wh ^ neg);
                            sts32(Bim_lo, rb, wl ^ neg);
                        }
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            f0[u] = cmul(f0[u], q0[u]);
                            q0[u].x *= g0;
                            q0[u].y *= g0;
                        }
                    }
                    // make the stores visible to the tensor cores, then hand the stage over
                    tc::fence_async_smem();
                }
                __syncwarp();
                if (lane == 0) {
                    hdr[s] = ok ? nvalid : 0;
                    bar_arrive(tc::smem_u32(full + s));
                }
            };
            // candidates of this warp: chunks of 32 records, round robin over the producers
            for (int64_t c0 = (int64_t)it.y + 32 * warp; c0 < it.z; c0 += 32 * PL_PROD) {
                const int64_t c = c0 + lane;
                bool kp = false;
                if (c < it.z) {
                    const float *qr = P.rec + c * REC;
                    const float g0d = fmaxf(fmaxf(blo0 - qr[0], qr[0] - bhi0), 0.f);
                    const float g1d = fmaxf(fmaxf(blo1 - qr[1], qr[1] - bhi1), 0.f);
                    const float g2d = P.x2 - qr[2];
                    kp = g0d * g0d + g1d * g1d + g2d * g2d <= P.rw2;
                }
                const unsigned bl = __ballot_sync(0xffffffffu, kp);
                if (kp) q[(qt + __popc(bl & ((1u << lane) - 1u))) & (PL_QUEUE - 1)] = (int)c;
                qt += __popc(bl);
                __syncwarp();
                if (qt - qh >= PL_KB) {
                    produce(PL_KB);
                    qh += PL_KB;
                    __syncwarp();
                }
            }
            if (qt > qh) produce(qt - qh);
            if (COUNT) {
                for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
                if (lane == 0 && pairs) atomicAdd(&g_plane_pairs, pairs);
            }
            // all producers done with the item: one END block closes its sequence
            asm volatile("bar.sync 1, %0;" ::"r"(PL_PROD * 32) : "memory");
            if (warp == 0) {
                int n = 0;
                if (lane == 0) n = atomicAdd(misc + 0, 1);
                n = __shfl_sync(0xffffffffu, n, 0);
                const int s = n % P.nst, use = n / P.nst;
                if (lane == 0) {
                    bool w = true;
                    if (use > 0 && *abort_flag == 0)
                        w = wait_taken(misc + 3, n - P.nst + 1, P.err) &&
                            bar_wait(tc::smem_u32(empty + s), (uint32_t)((use - 1) & 1), P.err);
                    if (!w) {
                        *abort_flag = 1;
                        report_timeout(P.err, 2, n, s, (use - 1) & 1, misc[0], misc[3]);
                    }
                    hdr[s] = -1;
                    bar_arrive(tc::smem_u32(full + s));
                }
                __syncwarp();
            }
        } else if (lane == 0) {
            // ------------------------------------------------ MMA issuer ---------------------------
            const uint32_t idesc = tc::instr_desc(NR, 128);
            bool started = false;
            for (;;) {
                const int s = mma_n % P.nst, use = mma_n / P.nst;
                mma_n++;
                bool w = bar_wait(tc::smem_u32(full + s), (uint32_t)(use & 1), P.err);
                if (!w) {
                    // no END will come in time: stop consuming (the producers time out as well)
                    *abort_flag = 1;
                    report_timeout(P.err, 3, mma_n - 1, s, use & 1, misc[0], misc[3]);
                    break;
                }
                *reinterpret_cast<volatile int *>(misc + 3) = mma_n;   // blocks taken so far
                const int nb = hdr[s];
                if (nb < 0) {
                    bar_arrive(tc::smem_u32(empty + s));   // the END block holds no data
                    break;
                }
                tc::fence_after();
                if (nb > 0 && *abort_flag == 0) {
                    const unsigned char *st = stages + s * P.stage_bytes;
                    const uint32_t a_base = tc::smem_u32(st), b_base = tc::smem_u32(st + 4 * PL_A_COPY);
                    for (int half = 0; half < 2; half++) {
                        const uint32_t a_hi = a_base + (2 * half) * PL_A_COPY, a_lo = a_hi + PL_A_COPY;
                        const uint32_t b_hi = b_base + (2 * half) * P.b_copy, b_lo = b_hi + P.b_copy;
                        for (int ks = 0; ks < PL_KB / 16; ks++) {
                            const uint32_t kof = ks * 2 * PL_LBO;
                            const uint64_t dah = tc::smem_desc_lbo_sbo(a_hi + kof, PL_LBO, PL_SBO_A);
                            const uint64_t dal = tc::smem_desc_lbo_sbo(a_lo + kof, PL_LBO, PL_SBO_A);
                            const uint64_t dbh = tc::smem_desc_lbo_sbo(b_hi + kof, PL_LBO, P.sbo_b);
                            const uint64_t dbl = tc::smem_desc_lbo_sbo(b_lo + kof, PL_LBO, P.sbo_b);
                            tc::mma_f16(tmem, dah, dbh, idesc, started ? 1u : 0u);
                            started = true;
                            tc::mma_f16(tmem, dah, dbl, idesc, 1u);
                            tc::mma_f16(tmem, dal, dbh, idesc, 1u);
                        }
                    }
                    tc::commit(tc::smem_u32(empty + s));
                } else {
                    bar_arrive(tc::smem_u32(empty + s));
                }
            }
            // every MMA of the item complete before the accumulator is read
            tc::commit(tc::smem_u32(done));
            if (!bar_wait(tc::smem_u32(done), done_par, P.err)) {
                *abort_flag = 1;
                report_timeout(P.err, 4, mma_n, 0, done_par, misc[0], misc[3]);
                tc::mbar_drain(tc::smem_u32(done), done_par);
            }
            done_par ^= 1u;
            misc[2] = started ? 1 : 0;
        }
        if (warp == PL_PROD) {
            // lanes 1..31 of the MMA warp follow lane 0's block counter
            mma_n = __shfl_sync(0xffffffffu, mma_n, 0);
            done_par = __shfl_sync(0xffffffffu, done_par, 0);
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- epilogue: TMEM lanes 0..63 (warps 0 and 1) -> the item's partial sums ----
        if (warp < 2) {
            const int row = 32 * warp + lane;
            const int tj = (row & 31) / 3, c = (row & 31) - 3 * tj, j = warp * J + tj;
            const bool have = misc[2] != 0 && *abort_flag == 0;
            const bool rowok = (row & 31) < 3 * J && j < e1;
            const float inv = 1.0f / (sa * sb);
            float *dst = P.partial + (int64_t)item * P.T0 * P.T1 * 6;
            for (int c0 = 0; c0 < P.nc; c0 += 8) {
                float re[8], im[8];
                if (have) {
                    tc::ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, re);
                    tc::ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(P.nc + c0), im);
                } else {
#pragma unroll
                    for (int u = 0; u < 8; u++) re[u] = im[u] = 0.f;
                }
                if (rowok) {
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int i = c0 + u;
                        if (i < P.T0) {
                            const int pnt = i * P.T1 + j;
                            dst[pnt * 6 + 2 * c] = re[u] * inv;
                            dst[pnt * 6 + 2 * c + 1] = im[u] * inv;
                        }
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    __syncthreads();
    if (warp == PL_PROD) tc::dealloc(tmem, P.tcols);
}

}  // namespace

// the plane kernel takes single-plane lattices with uniform axes 0 and 1
bool plane_tc_eligible(const LatticePlan &plan) {
    return plan.n[2] == 1 && plan.T[2] == 1 && (plan.uniform[0] || plan.n[0] == 1) &&
           (plan.uniform[1] || plan.n[1] == 1) && plan.T[0] <= PL_T0_MAX && plan.T[1] <= PL_T1_MAX;
}

void tile_shape_plane(const fga_lattice &L, int T[3]) {
    T[2] = 1;
    const int nt1 = (L.n[1] + PL_T1_MAX - 1) / PL_T1_MAX;
    T[1] = (L.n[1] + nt1 - 1) / nt1;
    const int nt0 = (L.n[0] + PL_T0_MAX - 1) / PL_T0_MAX;
    T[0] = (L.n[0] + nt0 - 1) / nt0;
}

fga_status run_plane_tc(Workspace &ws, const LatticePlan &plan, const void *rec, double k, double rw, void *u,
                        cudaStream_t s, int cat) {
    const int T0 = plan.T[0], T1 = plan.T[1];
    const int TP = T0 * T1;
    const int nc = (T0 + 7) / 8 * 8;
    // row-group stride of the B copies: the Re rows (i) and Im rows (nc + i) stored by the two lane
    // halves in one instruction land 16 banks apart
    int sbo_b = 576;
    while (((nc / 8) * sbo_b) % 128 != 64) sbo_b += 16;
    const int b_copy = (2 * nc / 8) * sbo_b;
    const int stage_bytes = (4 * PL_A_COPY + 4 * b_copy + 1023) / 1024 * 1024;
    const int extra = PL_A_COPY + 2 * PL_STAGES * 8 + 8 + PL_STAGES * 4 + 8 * 4 + PL_PROD * PL_QUEUE * 4 + 64;
    const int nst = std::min(PL_STAGES, (227 * 1024 - extra) / stage_bytes);
    const int bytes = nst * stage_bytes + extra;
    if (nst < 2) {
        set_error("plane tile does not fit the tensor-core plane kernel");
        return FGA_ERR_UNSUPPORTED;
    }
    FGA_TRY(ws.partial.ensure(sizeof(float) * 6 * (size_t)TP * (size_t)std::max(plan.nitems, 1) + 64));
    char *tailp = ws.partial.as<char>() + sizeof(float) * 6 * (size_t)TP * (size_t)std::max(plan.nitems, 1);
    float *amax = reinterpret_cast<float *>(tailp);
    FGA_CUDA(cudaMemsetAsync(tailp, 0, 64, s));
    if (!ws.status.p) FGA_TRY(status_reset(ws, s));
    prof_add_pairs_tested(plan.pairs_tested);
    if (plan.nitems > 0) {
        FGA_TRY(rec_absmax(static_cast<const float *>(rec), plan.n_rec, amax, s, cat));
        PlaneArgs A;
        A.rec = static_cast<const float *>(rec);
        A.items = plan.items;
        A.nitems = plan.nitems;
        A.n0 = plan.n[0];
        A.n1 = plan.n[1];
        A.T0 = T0;
        A.T1 = T1;
        A.nt1 = plan.nt[1];
        A.nc = nc;
        A.sbo_b = sbo_b;
        A.b_copy = b_copy;
        A.stage_bytes = stage_bytes;
        A.nst = nst;
        A.x0 = (float)plan.x_first[0];
        A.h0 = (float)plan.dx[0];
        A.x1 = (float)plan.x_first[1];
        A.h1 = (float)plan.dx[1];
        A.x2 = (float)plan.x_first[2];
        A.k = (float)k;
        A.rw2 = (float)(rw * rw);
        A.amax = amax;
        A.partial = ws.partial.as<float>();
        A.err = ws.status.as<int>();
        A.tcols = 2 * nc <= 32 ? 32u : (2 * nc <= 64 ? 64u : 128u);
        int dev = 0, sms = 152;
        FGA_CUDA(cudaGetDevice(&dev));
        FGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = std::min(plan.nitems, sms);
        ProfScope ps(cat, s);
        if (prof_counting()) {
            FGA_CUDA(cudaFuncSetAttribute(plane_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            plane_tc_kernel<true><<<grid, PL_THREADS, bytes, s>>>(A);
        } else {
            FGA_CUDA(cudaFuncSetAttribute(plane_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
            plane_tc_kernel<false><<<grid, PL_THREADS, bytes, s>>>(A);
        }
        FGA_CUDA(cudaGetLastError());
    }
    FGA_TRY(lattice_reduce_f32(ws.partial.as<float>(), plan, u, s));
    return FGA_OK;
}

}  // namespace fga
