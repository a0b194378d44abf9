// A6 on single-plane lattices (receiver arrays: n0 x n1 points at one x3), FP32 path, on the
// tensor cores with warp-specialised producers.
//
// On a tile of T0 x T1 points of the plane, with E_d the per-axis Gaussian factors of Eq. FGA,
//
//   U[(j,c)][i] = sum_b  W_bc E1_b(x_j) E0_b(x_i),      W_bc = A_bc E2_b(x_2)
//
// is a complex matrix product over the beams b (the contraction index): rows (j, c) -> TMEM lanes
// r = 32 h + 3 t + c with j = h J + t (J = ceil(T1/2), h in {0, 1}), columns i.  One B operand
// B' = [Re E0; Im E0] serves both halves of the complex product: A_re B'^T and A_im B'^T go to two
// accumulators, and Re U = A_re Re E0 - A_im Im E0, Im U = A_re Im E0 + A_im Re E0 are formed in the
// epilogue.
// Both operands are FP16 hi/lo splits of the FP32 values (hi*hi + hi*lo + lo*hi, FP32 accumulation),
// as in the other tensor-core kernels of the library.
//
// One persistent CTA per SM: seven producer warps and one MMA warp.
//  - Each producer warp owns one shared-memory stage.  It filters its share of an item's candidate
//    records (the beams within the window radius of the tile's box; four chunks of 32 in flight) into a
//    queue and turns every 32 kept beams into one operand block: lane (h, p) takes beams 2p and 2p+1,
//    forms W, E1 by recurrence on its half of the rows and E0 by a stride-2 recurrence on its parity
//    (the other parity comes from lane p + 16(1-h) by a shuffle), all in registers, then waits for its
//    stage and writes 32-bit pairs of FP16 values straight into the K-major operand layout.  The layout
//    is padded (leading byte offset 144, row-group stride chosen per tile) so that these stores are
//    free of bank conflicts.
//  - Per stage a "full" mbarrier (producer -> MMA) and an "empty" one (tcgen05.commit -> producer).
//    With one producer per stage every parity wait is exactly one phase behind the barrier.
//  - The MMA warp's elected thread takes the producers' blocks in a fixed cyclic order (so the
//    accumulation order, and the result, do not depend on timing) and issues four tcgen05.mma per block
//    (two K steps x re/im): each multiplies [A_hi; A_lo] (M = 128) by [B_hi; B_lo] (N = 4 n_c) into the
//    re or the im accumulator, so one instruction forms the three split products hi*hi, hi*lo and lo*hi
//    (and an unused lo*lo quarter); a tcgen05.mma costs about the same for N = 48 as for N = 96, so
//    fewer, wider instructions win.
//  - A producer closes its part of an item with an END block (no data); once every producer has, the
//    last commit is awaited and the accumulator rows go to the plan's per-item partial sums, reduced as
//    for the other lattice kernels.
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

constexpr int PL_PROD = 7;                     // producer warps, one shared-memory stage each
constexpr int PL_THREADS = (PL_PROD + 1) * 32; // + the MMA warp
constexpr int PL_KB = 32;                      // beams per block
constexpr int PL_LBO = 144;                    // bytes between K-adjacent core matrices
constexpr int PL_SBO_A = 592;                  // bytes between row-adjacent core matrices of A
constexpr int PL_A_COPY = 8 * PL_SBO_A;        // one A copy: 64 rows (8 row groups)
constexpr int PL_QUEUE = 64;                   // kept records queued per producer warp (31 + 32 used)
constexpr int PL_T0_MAX = 24, PL_T1_MAX = 20;   // seven 28 KB stages fit with n_c <= 24
constexpr int PL_PARK = 257;                   // floats per accumulator lane in the epilogue's copy

struct PlaneArgs {
    const float *rec;        // records [n_rec][12]: Q, P, weighted polarised amplitude (3 complex)
    const int4 *items;       // (tile, first record, end record, 0)
    int nitems;
    int n0, n1;              // lattice extents (n2 = 1)
    int T0, T1, nt1;         // tile shape and tiles along axis 1
    int nc;                  // complex accumulator columns (T0 rounded up to 8)
    int sbo_b;               // row-group stride of the B copies
    int b_copy, stage_bytes;
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

// the same split of a packed pair, the residual by one packed subtraction
__device__ __forceinline__ void split2p(float2 v, uint32_t &hi, uint32_t &lo) {
    const __half2 hh = __float22half2_rn(v);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __float22half2_rn(__fadd2_rn(v, make_float2(-hf.x, -hf.y)));
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

// row-group stride of the B copies for n_c complex columns: the Re rows (i) and the Im rows (n_c + i),
// stored by the two lane halves in one instruction, land 16 banks apart
__host__ __device__ constexpr int plane_sbo_b(int nc) {
    int sbo = 576;
    while (((nc / 8) * sbo) % 128 != 64) sbo += 16;
    return sbo;
}

// JT, T0T: the tile's j values per row half and points along axis 0 as compile-time constants (the
// loops over rows and points unroll, operand offsets become immediates); 0 = taken from the launch
template <bool COUNT, int JT, int T0T>
__global__ void __launch_bounds__(PL_THREADS, 1) plane_tc_kernel(PlaneArgs P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *tail = smem + PL_PROD * P.stage_bytes + PL_A_COPY;
    uint64_t *full = reinterpret_cast<uint64_t *>(tail);
    uint64_t *empty = full + PL_PROD;
    uint64_t *done = empty + PL_PROD;
    int *hdr = reinterpret_cast<int *>(done + 1);          // per stage: beams in the block, -1 = END
    int *misc = hdr + PL_PROD;                             // 1 abort, 2 item had MMAs, 3 blocks taken
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(misc + 4);
    float4 *queues = reinterpret_cast<float4 *>(tail + 256);  // [PL_PROD][PL_QUEUE][3]: kept records

    if (warp == PL_PROD) tc::alloc(tc::smem_u32(tmem_slot), P.tcols);
    if (tid == 0) {
        for (int s = 0; s < PL_PROD; s++) {
            tc::mbar_init(tc::smem_u32(full + s));
            tc::mbar_init(tc::smem_u32(empty + s));
        }
        tc::mbar_init(tc::smem_u32(done));
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

    const int J = JT ? JT : (P.T1 + 1) >> 1;         // j values per row half
    const int T0 = T0T ? T0T : P.T0;
    const int NC = T0T ? (T0T + 7) / 8 * 8 : P.nc;
    const int SBOB = T0T ? plane_sbo_b((T0T + 7) / 8 * 8) : P.sbo_b;
    const float hk = -0.5f * P.k;
    uint32_t done_par = 0;
    int uses = 0;                            // producer: fills of its stage so far (never reset)
    uint32_t fullpar = 0;                    // MMA thread: bit w = parity of stage w's next full phase

    for (int item = blockIdx.x; item < P.nitems; item += gridDim.x) {
        const int4 it = P.items[item];
        const int t = it.x, tt0 = t / P.nt1, tt1 = t % P.nt1;
        const int i0 = tt0 * T0, j0 = tt1 * P.T1;
        const int e0 = min(T0, P.n0 - i0), e1 = min(P.T1, P.n1 - j0);
        // the tile's box (window test of the candidates)
        const float blo0 = P.x0 + P.h0 * i0, bhi0 = P.x0 + P.h0 * (i0 + e0 - 1);
        const float blo1 = P.x1 + P.h1 * j0, bhi1 = P.x1 + P.h1 * (j0 + e1 - 1);
        if (warp < PL_PROD) {
            // ------------------------------------------------ producers ----------------------------
            const int w = warp;
            float4 *q = queues + w * PL_QUEUE * 3;
            int qh = 0, qt = 0;
            const int h = lane >> 4, p = lane & 15;
            unsigned long long pairs = 0;
            unsigned char *st = smem + w * P.stage_bytes;
            unsigned char *Are = st, *Are_lo = st + PL_A_COPY, *Aim = st + 2 * PL_A_COPY, *Aim_lo = st + 3 * PL_A_COPY;
            unsigned char *Bre = st + 4 * PL_A_COPY, *Bre_lo = Bre + P.b_copy;
            // wait until the MMAs of this stage's previous block are done (exactly one phase back)
            auto acquire = [&](int site, int n) -> bool {
                bool ok = *abort_flag == 0;
                if (uses > 0 && ok) {
                    bool wt = true;
                    if (lane == 0) wt = bar_wait(tc::smem_u32(empty + w), (uint32_t)((uses - 1) & 1), P.err);
                    wt = __shfl_sync(0xffffffffu, wt ? 1 : 0, 0) != 0;
                    if (!wt) {
                        if (lane == 0) {
                            *abort_flag = 1;
                            report_timeout(P.err, site, n, w, (uses - 1) & 1, uses, misc[3]);
                        }
                        ok = false;
                    }
                }
                return ok;
            };
            auto release = [&](int value) {
                __syncwarp();
                if (lane == 0) {
                    hdr[w] = value;
                    bar_arrive(tc::smem_u32(full + w));
                }
                uses++;
            };
            auto produce = [&](int nvalid) {
                // factors of the lane's two beams, in registers, before the stage is needed
                float2 W[2][3];
                float2 f1[2], q1[2], f0[2], q0[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int slot = 2 * p + u;
                    float r[REC];
                    if (slot < nvalid) {
                        const float4 *src = q + ((qh + slot) & (PL_QUEUE - 1)) * 3;
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
                const float g1 = __expf(-P.k * P.h1 * P.h1);
                const float g0 = __expf(-4.f * P.k * P.h0 * P.h0);
                const bool ok = acquire(1, uses);
                if (ok) {
                    // ---- A: rows r = 32 h + 3 t + c, j = h J + t ----
                    const uint32_t lanek = koff(0, 2 * p, 0) + (uint32_t)(h * 4 * PL_SBO_A);
                    // the lane's two beams side by side in packed FP32x2 registers: (beam 0, beam 1)
                    float2 Wr[3], Wi[3];
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        Wr[c] = make_float2(W[0][c].x, W[1][c].x);
                        Wi[c] = make_float2(-W[0][c].y, -W[1][c].y);   // negated: re = Wr F - Wi' ...
                    }
                    float2 Fr = make_float2(f1[0].x, f1[1].x), Fi = make_float2(f1[0].y, f1[1].y);
                    float2 Qr = make_float2(q1[0].x, q1[1].x), Qi = make_float2(q1[0].y, q1[1].y);
                    const float2 G1 = make_float2(g1, g1);
#pragma unroll
                    for (int tj = 0; tj < (JT ? JT : J); tj++) {
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const int row = 3 * tj + c;   // within the half (the half's 32 rows = 4 row groups)
                            // v = W F: re = Wr Fr - Wi Fi, im = Wr Fi + Wi Fr (Wi held negated)
                            const float2 vr = __ffma2_rn(Wi[c], Fi, __fmul2_rn(Wr[c], Fr));
                            const float2 vi = __ffma2_rn(make_float2(-Wi[c].x, -Wi[c].y), Fr, __fmul2_rn(Wr[c], Fi));
                            uint32_t rh, rl, ih, il;
                            split2p(vr, rh, rl);
                            split2p(vi, ih, il);
                            const uint32_t o = lanek + (uint32_t)((row >> 3) * PL_SBO_A + (row & 7) * 16);
                            sts32(Are, o, rh);
                            sts32(Are_lo, o, rl);
                            sts32(Aim, o, ih);
                            sts32(Aim_lo, o, il);
                        }
                        // F <- F Q, Q <- Q g1 (both beams at once)
                        const float2 nr = __ffma2_rn(make_float2(-Fi.x, -Fi.y), Qi, __fmul2_rn(Fr, Qr));
                        const float2 ni = __ffma2_rn(Fi, Qr, __fmul2_rn(Fr, Qi));
                        Fr = nr;
                        Fi = ni;
                        Qr = __fmul2_rn(Qr, G1);
                        Qi = __fmul2_rn(Qi, G1);
                    }
                    // ---- B: B' = [Re E0; Im E0]; half 0 stores the Re words, half 1 the Im words; each half
                    // forms E0 on its parity and gets the other one ----
                    const uint32_t lanekb = koff(0, 2 * p, 0);
                    const uint32_t rowoff_a = h == 0 ? 0u : (uint32_t)((NC >> 3) * SBOB);   // Re rows | Im rows
#pragma unroll
                    for (int i2 = 0; i2 < (T0T ? T0T : T0); i2 += 2) {
                        float2 mine[2] = {f0[0], f0[1]}, other[2];
#pragma unroll
                        for (int u = 0; u < 2; u++) {
                            other[u].x = __shfl_xor_sync(0xffffffffu, mine[u].x, 16);
                            other[u].y = __shfl_xor_sync(0xffffffffu, mine[u].y, 16);
                        }
#pragma unroll
                        for (int par = 0; par < 2; par++) {
                            const int i = i2 + par;
                            if (i >= (T0T ? T0T : T0)) break;
                            const float2 v0 = (par == h) ? mine[0] : other[0];
                            const float2 v1 = (par == h) ? mine[1] : other[1];
                            uint32_t wh, wl;
                            split2(h == 0 ? v0.x : v0.y, h == 0 ? v1.x : v1.y, wh, wl);
                            const uint32_t ra = lanekb + (uint32_t)((i >> 3) * SBOB + (i & 7) * 16) + rowoff_a;
                            sts32(Bre, ra, wh);
                            sts32(Bre_lo, ra, wl);
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
                release(ok ? nvalid : 0);
            };
            // candidates of this producer: chunks of 32 records dealt round robin over the producers; the
            // next chunk's records are loaded (coalesced, one record per lane) while this one is filtered and
            // its kept records are queued in shared memory and turned into blocks
            const int64_t stride = 32 * PL_PROD;
            int64_t c0 = (int64_t)it.y + 32 * w;
            float4 na = make_float4(0.f, 0.f, 0.f, 0.f), nb = na, nc = na;
            if (c0 + lane < it.z) {
                const float4 *src = reinterpret_cast<const float4 *>(P.rec + (c0 + lane) * REC);
                na = src[0];
                nb = src[1];
                nc = src[2];
            }
            for (; c0 < it.z; c0 += stride) {
                const float4 ra = na, rb = nb, rc = nc;
                const int64_t c = c0 + lane, cn = c + stride;
                if (cn < it.z) {
                    const float4 *src = reinterpret_cast<const float4 *>(P.rec + cn * REC);
                    na = src[0];
                    nb = src[1];
                    nc = src[2];
                }
                bool kp = false;
                if (c < it.z) {
                    const float g0d = fmaxf(fmaxf(blo0 - ra.x, ra.x - bhi0), 0.f);
                    const float g1d = fmaxf(fmaxf(blo1 - ra.y, ra.y - bhi1), 0.f);
                    const float g2d = P.x2 - ra.z;
                    kp = g0d * g0d + g1d * g1d + g2d * g2d <= P.rw2;
                }
                const unsigned bl = __ballot_sync(0xffffffffu, kp);
                if (kp) {
                    float4 *dst = q + ((qt + __popc(bl & ((1u << lane) - 1u))) & (PL_QUEUE - 1)) * 3;
                    dst[0] = ra;
                    dst[1] = rb;
                    dst[2] = rc;
                }
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
            // this producer's part of the item is complete
            acquire(2, uses);
            release(-1);
        } else if (lane == 0) {
            // ------------------------------------------------ MMA issuer ---------------------------
            const uint32_t idesc = tc::instr_desc(256, 128);
            bool started = false;
            unsigned active = (1u << PL_PROD) - 1u;
            for (int w = 0; active != 0u; w = (w + 1 == PL_PROD) ? 0 : w + 1) {
                if (!((active >> w) & 1u)) continue;
                const uint32_t par = (fullpar >> w) & 1u;
                if (!bar_wait(tc::smem_u32(full + w), par, P.err)) {
                    *abort_flag = 1;
                    report_timeout(P.err, 3, misc[3], w, (int)par, 0, misc[3]);
                    break;
                }
                fullpar ^= 1u << w;
                misc[3]++;
                const int nb = hdr[w];
                if (nb < 0) {
                    active &= ~(1u << w);
                    bar_arrive(tc::smem_u32(empty + w));   // the END block holds no data
                    continue;
                }
                tc::fence_after();
                if (nb > 0 && *abort_flag == 0) {
                    const unsigned char *st = smem + w * P.stage_bytes;
                    const uint32_t a_base = tc::smem_u32(st), b_base = tc::smem_u32(st + 4 * PL_A_COPY);
                    // one M = 128 x N = 256 MMA per K step: accumulator lane m = row of [B'_hi; B'_lo] (lanes
                    // 0..63: Re E0 at i, Im E0 at n_c + i, hi; lanes 64..127 the same, lo), column n = row of
                    // the A copies (0..63 A_re hi, 64..127 A_re lo, 128..191 A_im hi, 192..255 A_im lo); the
                    // products lo*lo and the padding rows are not used
                    for (int ks = 0; ks < PL_KB / 16; ks++) {
                        const uint32_t kof = ks * 2 * PL_LBO;
                        // M side: the B copies [B'_hi; B'_lo] (64 rows each); N side: the four A copies
                        // [A_re_hi; A_re_lo; A_im_hi; A_im_lo] (64 rows each, one row-group stride)
                        const uint64_t dm = tc::smem_desc_lbo_sbo(b_base + kof, PL_LBO, SBOB);
                        const uint64_t dn = tc::smem_desc_lbo_sbo(a_base + kof, PL_LBO, PL_SBO_A);
                        tc::mma_f16(tmem, dm, dn, idesc, started ? 1u : 0u);
                        started = true;
                    }
                    tc::commit(tc::smem_u32(empty + w));
                } else {
                    bar_arrive(tc::smem_u32(empty + w));
                }
            }
            // every MMA of the item complete before the accumulator is read
            tc::commit(tc::smem_u32(done));
            if (!bar_wait(tc::smem_u32(done), done_par, P.err)) {
                *abort_flag = 1;
                report_timeout(P.err, 4, misc[3], 0, (int)done_par, 0, misc[3]);
                tc::mbar_drain(tc::smem_u32(done), done_par);
            }
            done_par ^= 1u;
            misc[2] = started ? 1 : 0;
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- epilogue: warps 0..3 copy their 32 accumulator lanes (all 256 columns) into the idle stage
        // memory, then every thread forms outputs U[(j,c)][i]:
        //   X_a(c', r) = hi*hi + hi*lo + lo*hi of A_a row r against E0 part c' (a, c' in {re, im})
        //   Re U = X_re(Re) - X_im(Im),  Im U = X_re(Im) + X_im(Re) ----
        const bool have = misc[2] != 0 && *abort_flag == 0;
        float *park = reinterpret_cast<float *>(smem);   // [128 lanes][PL_PARK] (padded rows: no bank conflicts)
        if (warp < 4) {
            const int ln = 32 * warp + lane;
            for (int c0 = 0; c0 < 256; c0 += 8) {
                float v[8];
                if (have) {
                    tc::ld8(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
                } else {
#pragma unroll
                    for (int u = 0; u < 8; u++) v[u] = 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; u++) park[ln * PL_PARK + c0 + u] = v[u];
            }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        {
            const float inv = 1.0f / (sa * sb);
            float *dst = P.partial + (int64_t)item * T0 * P.T1 * 6;
            const int nout = T0 * 2 * J * 3;   // (i, half, t, c)
            for (int o = tid; o < nout; o += PL_THREADS) {
                const int c = o % 3, t = (o / 3) % J, hh = (o / (3 * J)) % 2, i = o / (6 * J);
                const int j = hh * J + t;
                if (j >= e1) continue;
                const int r = 32 * hh + 3 * t + c;   // A row
                // x[a][p]: A_a (a: 0 re, 1 im) against Re E0 (p = 0) or Im E0 (p = 1)
                float x[2][2];
#pragma unroll
                for (int a2 = 0; a2 < 2; a2++)
#pragma unroll
                    for (int p2 = 0; p2 < 2; p2++) {
                        const int lhi = p2 * NC + i, llo = 64 + lhi;
                        const int chi = 128 * a2 + r, clo = chi + 64;
                        x[a2][p2] = park[lhi * PL_PARK + chi] + park[lhi * PL_PARK + clo] + park[llo * PL_PARK + chi];
                    }
                const int pnt = i * P.T1 + j;
                dst[pnt * 6 + 2 * c] = (x[0][0] - x[1][1]) * inv;
                dst[pnt * 6 + 2 * c + 1] = (x[0][1] + x[1][0]) * inv;
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
                        cudaStream_t s, int cat, const float *amax_in) {
    const int T0 = plan.T[0], T1 = plan.T[1];
    const int TP = T0 * T1;
    const int nc = (T0 + 7) / 8 * 8;
    // row-group stride of the B copies: the Re rows (i) and Im rows (nc + i) stored by the two lane
    // halves in one instruction land 16 banks apart
    const int sbo_b = plane_sbo_b(nc);
    const int b_copy = 8 * sbo_b;   // 64 rows: Re E0 (n_c), Im E0 (n_c), padding
    const int stage_bytes = (4 * PL_A_COPY + 2 * b_copy + 1023) / 1024 * 1024;
    const int bytes = PL_PROD * stage_bytes + PL_A_COPY + 256 + PL_PROD * PL_QUEUE * 48;
    if (bytes > 227 * 1024) {
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
        if (!amax_in) FGA_TRY(rec_absmax(static_cast<const float *>(rec), plan.n_rec, amax, s, cat));
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
        A.x0 = (float)plan.x_first[0];
        A.h0 = (float)plan.dx[0];
        A.x1 = (float)plan.x_first[1];
        A.h1 = (float)plan.dx[1];
        A.x2 = (float)plan.x_first[2];
        A.k = (float)k;
        A.rw2 = (float)(rw * rw);
        A.amax = amax_in ? amax_in : amax;
        A.partial = ws.partial.as<float>();
        A.err = ws.status.as<int>();
        // the accumulator: 128 lanes x 256 columns
        A.tcols = 256u;
        int dev = 0, sms = 152;
        FGA_CUDA(cudaGetDevice(&dev));
        FGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = std::min(plan.nitems, sms);
        ProfScope ps(cat, s);
        const int J = (T1 + 1) / 2;
        const bool cnt = prof_counting();
#define FGA_PLANE(CNT, JT, T0T)                                                                                   \
    do {                                                                                                          \
        FGA_CUDA(cudaFuncSetAttribute(plane_tc_kernel<CNT, JT, T0T>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      bytes));                                                                    \
        plane_tc_kernel<CNT, JT, T0T><<<grid, PL_THREADS, bytes, s>>>(A);                                         \
    } while (0)
        // the receiver planes of the benchmark (20 x 20) and of the serving mix (16 x 16) unrolled
        if (J == 10 && T0 == 20) {
            if (cnt) FGA_PLANE(true, 10, 20);
            else FGA_PLANE(false, 10, 20);
        } else if (J == 8 && T0 == 16) {
            if (cnt) FGA_PLANE(true, 8, 16);
            else FGA_PLANE(false, 8, 16);
        } else {
            if (cnt) FGA_PLANE(true, 0, 0);
            else FGA_PLANE(false, 0, 0);
        }
#undef FGA_PLANE
        FGA_CUDA(cudaGetLastError());
    }
    FGA_TRY(lattice_reduce_f32(ws.partial.as<float>(), plan, u, s));
    return FGA_OK;
}

}  // namespace fga
