// A6 on tensor lattices (receiver arrays, snapshot grids), FP32 path, on the tensor cores.
//
// With E_d(x) = exp(i k P_d (x - Q_d) - k (x - Q_d)^2 / 2) the Gaussian of Eq. FGA factors per axis,
// so on a tile of T0 x T1 x T2 lattice points the sum over the beams b of a tile's neighbourhood is a
// complex matrix product with the beams as the contraction index:
//
//   U[(j,l)][(i,c)] = sum_b  Y_b[(j,l)] X_b[(i,c)],   Y_b[(j,l)] = E1_b(x_j) E2_b(x_l),
//                                                   X_b[(i,c)] = A_bc E0_b(x_i)
//
// (A_bc: component c of the beam's weighted polarised amplitude).  Per block of 32 beams the CUDA
// cores form the 1-D factors (on an axis with uniform spacing h by the recurrence E(x + h) = E(x) R(x),
// R(x + h) = R(x) exp(-k h^2), restarted with two exponentials every 8 points; else one exponential
// per point) and the two operand blocks (T1 T2 + 3 T0 complex values per beam) instead of one complex
// product per point and component; the 5th-generation tensor cores do the T1 T2 x 3 T0 x 32 product in FP16 split precision
// (hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory), like the transform of A1.  Every
// (beam, point) pair of the binned neighbourhood is summed: the pairs beyond the window radius carry
// a Gaussian below e^-18 and change the sum by less than e^-18 of sum |A|.
//
// One CTA = one work item (tile, range of cell-sorted records) of the lattice plan; 256 threads, two
// CTAs per SM (the tensor cores of one overlap the operand formation of the other).
// Rows (j,l) of the tile are the 128 TMEM lanes (M = 128; unused rows stay zero), columns are
// Re/Im of the 3 T0 complex (i,c) pairs.  Operand blocks are single-buffered: the records and factors
// of the next block are formed while the tensor cores work on the current one.  The partial sums go
// to the plan's per-item buffer in the layout of the CUDA-core lattice kernel and are reduced by it.
#include <algorithm>
#include <cstdio>
#include <cmath>

#include "fga_beam.cuh"
#include "gather.cuh"
#include "tcgen05.cuh"

namespace fga {

// (beam, point) pairs inside the window (profiling)
static __device__ unsigned long long g_tc_pairs;

int64_t read_tc_pair_counter(bool reset) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_pairs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_tc_pairs, &z, sizeof z);
    }
    return (int64_t)v;
}

namespace {

constexpr int LT_M = 128;
constexpr int LT_THREADS = 256;
constexpr int LT_CHUNK = 8;              // points per factor recurrence on a uniform axis
constexpr int LT_KB = tc::KB;            // beams per block
constexpr int LT_T0_MAX = 32;            // 6 T0 <= 192 real columns
constexpr int LT_NMAX = 192;
constexpr int LT_A_BYTES = LT_M * LT_KB * 2;      // 8 KB per operand copy
constexpr int LT_TA_MAX = 32 + 128 + 16;
constexpr int LT_CAND = 4096;           // candidates filtered per round (per-CTA kept-list scratch)

// shared-memory layout; the B operand copies and the tensor-memory columns are sized to the tile's
// real width NR, so narrow tiles (single receiver planes) fit three CTAs per SM
struct LtSmem {
    int a, b, e, rec, w, x, cnt, bar, bytes, bbytes;
    uint32_t tcols;
    __host__ __device__ void init(int TA, bool with_w, int NR) {
        bbytes = NR * LT_KB * 2;
        tcols = NR <= 32 ? 32u : (NR <= 64 ? 64u : (NR <= 128 ? 128u : 256u));
        a = 0;
        b = a + 4 * LT_A_BYTES;
        e = b + 4 * bbytes;                     // 2 x [32][TA] float2
        rec = e + 2 * LT_KB * TA * 8;           // 2 x [32][REC] float
        w = rec + 2 * LT_KB * REC * 4;          // 2 x [32][3] float2: A_c E2 of single-plane tiles
        x = w + (with_w ? 2 * LT_KB * 3 * 8 : 0);
        cnt = (x + TA * 4 + 15) / 16 * 16;
        bar = cnt + (LT_THREADS / 32 + 1) * 4;
        bar = (bar + 15) / 16 * 16;
        bytes = bar + 16;
    }
};

// per-axis factor chunks: uniform axes in runs of LT_CHUNK points (one exponential for the first point
// and one for the ratio, then E <- E R, R <- R G with G = exp(-k dx^2)), other axes point by point
struct LtAxes {
    int len[3];    // points per chunk
    int nch[3];    // chunks per axis
    float dx[3];   // spacing of uniform axes
};

// Operand mapping.  crow = 0: rows (j, l), columns (i, c): Y = E1 E2, X = A_c E0.
//                  crow = 1 (small T1 T2): rows (j, l, c), columns i: Y = A_c E1 E2, X = E0.
template <bool COUNT, int MINB>
__global__ void __launch_bounds__(LT_THREADS, MINB) lattice_tc_kernel(const float *__restrict__ rec, const double *__restrict__ ax0,
                                                        const double *__restrict__ ax1, const double *__restrict__ ax2,
                                                        int n0, int n1, int n2, int T0, int T1, int T2, int nt1,
                                                        int nt2, const int4 *__restrict__ items, float k, float rw2,
                                                        const float *__restrict__ amax, LtSmem S, LtAxes X, int crow,
                                                        int *__restrict__ kept, float *__restrict__ partial,
                                                        int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem + S.a;
    unsigned char *sB = smem + S.b;
    float2 *sE0 = reinterpret_cast<float2 *>(smem + S.e);   // 2 x [32][TA]: E0 (T0), E1 (T1), E2 (T2)
    float *sR0 = reinterpret_cast<float *>(smem + S.rec);   // 2 x [32][REC]
    float2 *sW0 = reinterpret_cast<float2 *>(smem + S.w);   // 2 x [32][3]
    float *sX = reinterpret_cast<float *>(smem + S.x);      // tile coordinates, axis 0 | 1 | 2
    int *sCnt = reinterpret_cast<int *>(smem + S.cnt);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S.bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    constexpr int NW = LT_THREADS / 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int TA = T0 + T1 + T2;
    const int R_used = crow ? 3 * T1 * T2 : T1 * T2, nc_used = crow ? T0 : 3 * T0;
    const int nc_tile = (nc_used + 7) / 8 * 8, NR = 2 * nc_tile;

    const int4 it = items[blockIdx.x];
    const int t = it.x;
    const int tt0 = t / (nt1 * nt2), tt1 = (t / nt2) % nt1, tt2 = t % nt2;
    const int i0 = tt0 * T0, j0 = tt1 * T1, l0 = tt2 * T2;
    const int e0 = min(T0, n0 - i0), e1 = min(T1, n1 - j0), e2 = min(T2, n2 - l0);

    const int LT_B_BYTES = S.bbytes;
    for (int o = tid * 16; o < 4 * LT_A_BYTES + 4 * LT_B_BYTES; o += LT_THREADS * 16)
        *reinterpret_cast<uint4 *>(smem + o) = make_uint4(0, 0, 0, 0);
    for (int a = tid; a < TA; a += LT_THREADS) {
        double v;
        if (a < T0) v = ax0[i0 + min(a, e0 - 1)];
        else if (a < T0 + T1) v = ax1[j0 + min(a - T0, e1 - 1)];
        else v = ax2[l0 + min(a - T0 - T1, e2 - 1)];
        sX[a] = (float)v;
    }
    if (warp == 0) tc::alloc(tc::smem_u32(tmem_slot), S.tcols);
    if (tid == 0) tc::mbar_init(tc::smem_u32(bar));
    float sx = 1.0f;
    {
        const float bound = *amax;
        if (bound > 0.0f && isfinite(bound)) {
            int e;
            frexpf(bound, &e);
            sx = ldexpf(1.0f, 14 - e);
        }
    }
    const float sy = 16384.0f;
    // the A_c factor carries the amplitude scale on whichever side it sits
    const float sA_scale = crow ? sx : sy, sB_scale = crow ? sy : sx;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::instr_desc(NR, LT_M);
    const float hk = -0.5f * k;
    // exact small-integer division by float reciprocals (quotients below 2^12, divisors below 2^8)
    const int nch = X.nch[0] + X.nch[1] + X.nch[2];
    const float inv_nch = 1.0f / (float)nch, inv_R = 1.0f / (float)R_used, inv_nc = 1.0f / (float)nc_used;
    const float inv_T2 = 1.0f / (float)T2, inv_3 = 1.0f / 3.0f;

    const float blo0 = sX[0], bhi0 = sX[e0 - 1], blo1 = sX[T0], bhi1 = sX[T0 + e1 - 1];
    const float blo2 = sX[T0 + T1], bhi2 = sX[T0 + T1 + e2 - 1];
    int *keptc = kept + (int64_t)blockIdx.x * LT_CAND;   // this CTA's kept list of one candidate round
    bool ok = true;
    uint32_t parity = 0;
    int issued = 0;
    for (int64_t cand0 = it.y; cand0 < it.z && ok; cand0 += LT_CAND) {
        // ---- 0. keep the round's candidates within rw of the tile's box, in order ----
        const int64_t cend = (it.z < cand0 + LT_CAND) ? (int64_t)it.z : cand0 + LT_CAND;
        int nk = 0;
        for (int64_t c0 = cand0; c0 < cend; c0 += LT_THREADS) {
            const int64_t c = c0 + tid;
            bool kp = false;
            if (c < cend) {
                const float *q = rec + c * REC;
                const float g0 = fmaxf(fmaxf(blo0 - q[0], q[0] - bhi0), 0.f);
                const float g1 = fmaxf(fmaxf(blo1 - q[1], q[1] - bhi1), 0.f);
                const float g2 = fmaxf(fmaxf(blo2 - q[2], q[2] - bhi2), 0.f);
                kp = g0 * g0 + g1 * g1 + g2 * g2 <= rw2;
            }
            const unsigned bl = __ballot_sync(0xffffffffu, kp);
            if (lane == 0) sCnt[warp] = __popc(bl);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < NW; w++) {
                const int v = sCnt[w];
                before += w < warp ? v : 0;
                total += v;
            }
            if (kp) keptc[nk + before + __popc(bl & ((1u << lane) - 1u))] = (int)(c - it.y);
            nk += total;
            __syncthreads();
        }
        const int nblk = (nk + LT_KB - 1) / LT_KB;

        auto load_records = [&](int blk, float *dst) {
            const int kb0 = blk * LT_KB, nb = min(LT_KB, nk - kb0);
            for (int q = tid; q < LT_KB * REC; q += LT_THREADS) {
                const int b = q / REC;
                dst[q] = b < nb ? rec[(it.y + keptc[kb0 + b]) * REC + (q - b * REC)] : 0.0f;
            }
        };
        auto factors = [&](int blk, const float *sR, float2 *sE, float2 *sW) {
            const int nb = min(LT_KB, nk - blk * LT_KB);
            for (int q = tid; q < LT_KB * nch; q += LT_THREADS) {
                const int b = (int)(((float)q + 0.5f) * inv_nch), c = q - b * nch;
                const int d = c < X.nch[0] ? 0 : (c < X.nch[0] + X.nch[1] ? 1 : 2);
                const int cc = c - (d == 0 ? 0 : (d == 1 ? X.nch[0] : X.nch[0] + X.nch[1]));
                const int off = d == 0 ? 0 : (d == 1 ? T0 : T0 + T1), Td = d == 0 ? T0 : (d == 1 ? T1 : T2);
                const int a0 = cc * X.len[d], a1 = min(a0 + X.len[d], Td);
                float2 *dst = sE + b * TA + off;
                const bool wfold = crow && d == 2 && T2 == 1;   // also A_c E2 for the component rows
                if (b >= nb) {
                    for (int a = a0; a < a1; a++) dst[a] = make_float2(0.f, 0.f);
                    if (wfold)
                        for (int c = 0; c < 3; c++) sW[b * 3 + c] = make_float2(0.f, 0.f);
                    continue;
                }
                const float Qd = sR[b * REC + d], Pd = sR[b * REC + 3 + d];
                const float x = sX[off + a0] - Qd;
                float er, ei;
                gauss_phase_exp<float>(k * Pd * x, hk * x * x, &er, &ei);
                dst[a0] = make_float2(er, ei);
                if (wfold)
                    for (int c = 0; c < 3; c++) {
                        const float ar = sR[b * REC + 6 + 2 * c], ai = sR[b * REC + 7 + 2 * c];
                        sW[b * 3 + c] = make_float2(ar * er - ai * ei, ar * ei + ai * er);
                    }
                if (a1 - a0 > 1) {
                    const float h = X.dx[d];
                    float rr, ri;
                    gauss_phase_exp<float>(k * Pd * h, -k * h * (x + 0.5f * h), &rr, &ri);
                    const float g = __expf(-k * h * h);
                    for (int a = a0 + 1; a < a1; a++) {
                        const float nr = er * rr - ei * ri, ni = er * ri + ei * rr;
                        er = nr;
                        ei = ni;
                        dst[a] = make_float2(er, ei);
                        rr *= g;
                        ri *= g;
                    }
                }
            }
            if (COUNT) {
                unsigned long long mine = 0;
                const int np = T0 * T1 * T2;
                for (int q = tid; q < nb * np; q += LT_THREADS) {
                    const int b = q / np, rem = q - b * np;
                    const int i = rem / (T1 * T2), r = rem - i * (T1 * T2), j = r / T2, l = r - j * T2;
                    if (i < e0 && j < e1 && l < e2) {
                        const float *rb = sR + b * REC;
                        const float d0 = sX[i] - rb[0], d1 = sX[T0 + j] - rb[1], d2 = sX[T0 + T1 + l] - rb[2];
                        if (d0 * d0 + d1 * d1 + d2 * d2 <= rw2) mine++;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
                if (lane == 0 && mine) atomicAdd(&g_tc_pairs, mine);
            }
        };

        // ---- software pipeline over the round's blocks of 32 kept beams ----
        // block n: operands from (sR, sE)[n % 2]; while the tensor cores run block n, the factors of
        // n+1 are formed and the records of n+2 loaded
        if (nblk > 0) load_records(0, sR0);
        __syncthreads();
        if (nblk > 0) factors(0, sR0, sE0, sW0);
        if (nblk > 1) load_records(1, sR0 + LT_KB * REC);
        for (int n = 0; n < nblk; n++) {
            const float *sR = sR0 + (n & 1) * LT_KB * REC;
            const float2 *sE = sE0 + (n & 1) * LT_KB * TA;
            bool arrived = true;
            if (issued > 0 && tid == 0) arrived = tc::mbar_wait(tc::smem_u32(bar), parity);
            ok = __syncthreads_and(arrived ? 1 : 0) != 0;   // factors(n) visible; the previous MMAs done
            tc::fence_after();
            if (!ok) break;
            if (issued > 0) parity ^= 1u;
        // operands: consecutive threads take consecutive rows (conflict-free 16-byte stores)
        const float2 *sW = sW0 + (n & 1) * LT_KB * 3;
        for (int q = tid; q < R_used * 4; q += LT_THREADS) {
            const int o = (int)(((float)q + 0.5f) * inv_R), r = q - o * R_used;
            float re[8], im[8];
            if (!crow) {
                const int j = (int)(((float)r + 0.5f) * inv_T2), l = r - j * T2;
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int b = 8 * o + u;
                    const float2 a1 = sE[b * TA + T0 + j], a2 = sE[b * TA + T0 + T1 + l];
                    re[u] = a1.x * a2.x - a1.y * a2.y;
                    im[u] = a1.x * a2.y + a1.y * a2.x;
                }
            } else {
                const int jl = (int)(((float)r + 0.5f) * inv_3), c = r - 3 * jl;
                if (T2 == 1) {
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int b = 8 * o + u;
                        const float2 e = sE[b * TA + T0 + jl], wv = sW[b * 3 + c];
                        re[u] = wv.x * e.x - wv.y * e.y;
                        im[u] = wv.x * e.y + wv.y * e.x;
                    }
                } else {
                    const int j = (int)(((float)jl + 0.5f) * inv_T2), l = jl - j * T2;
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int b = 8 * o + u;
                        const float2 a1 = sE[b * TA + T0 + j], a2 = sE[b * TA + T0 + T1 + l];
                        const float er = a1.x * a2.x - a1.y * a2.y, ei = a1.x * a2.y + a1.y * a2.x;
                        const float ar = sR[b * REC + 6 + 2 * c], ai = sR[b * REC + 7 + 2 * c];
                        re[u] = ar * er - ai * ei;
                        im[u] = ar * ei + ai * er;
                    }
                }
            }
            const uint32_t off = tc::kmaj_off(r, 8 * o);
            tc::split8(sA + 0 * LT_A_BYTES, sA + 1 * LT_A_BYTES, off, re, sA_scale);
            tc::split8(sA + 2 * LT_A_BYTES, sA + 3 * LT_A_BYTES, off, im, sA_scale);
        }
        for (int q = tid; q < nc_used * 4; q += LT_THREADS) {
            const int o = (int)(((float)q + 0.5f) * inv_nc), cq = q - o * nc_used;
            float re[8], im[8], nim[8];
            if (!crow) {
                const int i = (int)(((float)cq + 0.5f) * inv_3), c = cq - 3 * i;
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int b = 8 * o + u;
                    const float2 e = sE[b * TA + i];
                    const float ar = sR[b * REC + 6 + 2 * c], ai = sR[b * REC + 7 + 2 * c];
                    re[u] = ar * e.x - ai * e.y;
                    im[u] = ar * e.y + ai * e.x;
                    nim[u] = -im[u];
                }
            } else {
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float2 e = sE[(8 * o + u) * TA + cq];
                    re[u] = e.x;
                    im[u] = e.y;
                    nim[u] = -e.y;
                }
            }
            const uint32_t top = tc::kmaj_off(cq, 8 * o), bot = tc::kmaj_off(nc_tile + cq, 8 * o);
            // B'_re = [Re X ; Im X], B'_im = [-Im X ; Re X]
            tc::split8(sB + 0 * LT_B_BYTES, sB + 1 * LT_B_BYTES, top, re, sB_scale);
            tc::split8(sB + 0 * LT_B_BYTES, sB + 1 * LT_B_BYTES, bot, im, sB_scale);
            tc::split8(sB + 2 * LT_B_BYTES, sB + 3 * LT_B_BYTES, top, nim, sB_scale);
            tc::split8(sB + 2 * LT_B_BYTES, sB + 3 * LT_B_BYTES, bot, re, sB_scale);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
            for (int half = 0; half < 2; half++) {
                const uint32_t a_hi = tc::smem_u32(sA + (2 * half) * LT_A_BYTES);
                const uint32_t a_lo = tc::smem_u32(sA + (2 * half + 1) * LT_A_BYTES);
                const uint32_t b_hi = tc::smem_u32(sB + (2 * half) * LT_B_BYTES);
                const uint32_t b_lo = tc::smem_u32(sB + (2 * half + 1) * LT_B_BYTES);
                for (int ks = 0; ks < LT_KB / 16; ks++) {
                    const uint32_t koff = ks * 2 * 128;
                    const uint32_t acc0 = (issued > 0 || half > 0 || ks > 0) ? 1u : 0u;
                    tc::mma_f16(tmem, tc::smem_desc(a_hi + koff), tc::smem_desc(b_hi + koff), idesc, acc0);
                    tc::mma_f16(tmem, tc::smem_desc(a_hi + koff), tc::smem_desc(b_lo + koff), idesc, 1u);
                    tc::mma_f16(tmem, tc::smem_desc(a_lo + koff), tc::smem_desc(b_hi + koff), idesc, 1u);
                }
            }
            tc::commit(tc::smem_u32(bar));
        }
        issued++;
        // while the tensor cores work: factors of block n+1, records of block n+2
        if (n + 1 < nblk)
            factors(n + 1, sR0 + ((n + 1) & 1) * LT_KB * REC, sE0 + ((n + 1) & 1) * LT_KB * TA,
                    sW0 + ((n + 1) & 1) * LT_KB * 3);
        if (n + 2 < nblk) load_records(n + 2, sR0 + (n & 1) * LT_KB * REC);
        }
        __syncthreads();   // the round's kept list and staging buffers are reused by the next round
    }
    if (ok && issued > 0) {
        bool arrived = true;
        if (tid == 0) arrived = tc::mbar_wait(tc::smem_u32(bar), parity);
        ok = __syncthreads_and(arrived ? 1 : 0) != 0;
        tc::fence_after();
    }
    // give-up: report, and let the outstanding commit (phase `parity`) land before freeing its columns
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        tc::mbar_drain(tc::smem_u32(bar), parity);
    }
    if (ok) {
        // epilogue: warps w and w + 4 share TMEM lanes 32 (w % 4) .. + 31 and split the 8-column chunks
        const int quarter = warp & 3, r = quarter * 32 + lane;
        const int TP = T0 * T1 * T2;
        const float inv = 1.0f / (sx * sy);
        float *dst = partial + (int64_t)blockIdx.x * TP * 6;
        const uint32_t lanebase = (uint32_t)(quarter * 32) << 16;
        for (int c0 = (warp >> 2) * 8; c0 < nc_tile; c0 += 16) {
            float re[8], im[8];
            if (issued > 0) {
                tc::ld8(tmem + lanebase + (uint32_t)c0, re);
                tc::ld8(tmem + lanebase + (uint32_t)(nc_tile + c0), im);
            } else {
#pragma unroll
                for (int u = 0; u < 8; u++) re[u] = im[u] = 0.f;
            }
            if (r < R_used) {
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const int cq = c0 + u;
                    if (cq < nc_used) {
                        int i, c, j, l;
                        if (!crow) {
                            i = cq / 3;
                            c = cq - 3 * i;
                            j = r / T2;
                            l = r - j * T2;
                        } else {
                            i = cq;
                            c = r % 3;
                            const int jl = r / 3;
                            j = jl / T2;
                            l = jl - j * T2;
                        }
                        const int p = (i * T1 + j) * T2 + l;
                        dst[p * 6 + 2 * c] = re[u] * inv;
                        dst[p * 6 + 2 * c + 1] = im[u] * inv;
                    }
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::dealloc(tmem, S.tcols);
}

__global__ void rec_absmax_kernel(const float *__restrict__ rec, int64_t n, float *__restrict__ out) {
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n * 6; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(rec[(i / 6) * REC + 6 + (i % 6)]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
}

}  // namespace

fga_status status_reset(Workspace &ws, cudaStream_t s) {
    FGA_TRY(ws.status.ensure(64));
    FGA_CUDA(cudaMemsetAsync(ws.status.p, 0, 64, s));
    return FGA_OK;
}

fga_status status_check(Workspace &ws, cudaStream_t s, const char *who) {
    if (!ws.status.p) {
        FGA_CUDA(cudaStreamSynchronize(s));
        return FGA_OK;
    }
    int v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    FGA_CUDA(cudaMemcpyAsync(v, ws.status.p, sizeof v, cudaMemcpyDeviceToHost, s));
    FGA_CUDA(cudaStreamSynchronize(s));
    if (v[0]) {
        std::string m = std::string(who) + ": a tensor-core wait of the Gaussian sum ran out";
        if (v[2]) {
            char buf[160];
            std::snprintf(buf, sizeof buf,
                          " (wait %d: block %d, stage %d, parity %d, %d blocks claimed, CTA %d, %d blocks taken by the MMA thread)", v[2],
                          v[3], v[4], v[5], v[6], v[7], v[8]);
            m += buf;
        }
        set_error(m);
        return FGA_ERR_TIMEOUT;
    }
    if (v[1]) {
        set_error(std::string(who) + ": non-finite values in the beam state or the results");
        return FGA_ERR_NUMERIC;
    }
    return FGA_OK;
}

template <typename R>
__global__ void nonfinite_kernel(const R *__restrict__ x, int64_t n, int *__restrict__ flag) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// beam state in structure-of-arrays form: field f of beam b at st[f * cap + b], b < nb
template <typename R>
__global__ void nonfinite_state_kernel(const R *__restrict__ st, int64_t cap, int64_t nb, int *__restrict__ flag) {
    const R *fld = st + (int64_t)blockIdx.y * cap;
    bool bad = false;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(fld[b]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

fga_status flag_nonfinite_state(Workspace &ws, const void *st, int64_t cap, int64_t nb, int nf, int precision,
                                cudaStream_t s) {
    if (nb <= 0 || !st) return FGA_OK;
    if (!ws.status.p) FGA_TRY(status_reset(ws, s));
    const dim3 grid((unsigned)std::min<int64_t>(64, (nb + 255) / 256), (unsigned)nf);
    int *flag = ws.status.as<int>() + 1;
    if (precision == FGA_PREC_FP64)
        nonfinite_state_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(st), cap, nb, flag);
    else
        nonfinite_state_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(st), cap, nb, flag);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

fga_status flag_nonfinite(Workspace &ws, const void *data, int64_t n, int precision, cudaStream_t s) {
    if (n <= 0 || !data) return FGA_OK;
    if (!ws.status.p) FGA_TRY(status_reset(ws, s));
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::min<int64_t>((int64_t)sms * 8, (n + 255) / 256);
    int *flag = ws.status.as<int>() + 1;
    if (precision == FGA_PREC_FP64)
        nonfinite_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double *>(data), n, flag);
    else
        nonfinite_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float *>(data), n, flag);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

fga_status rec_absmax(const float *rec, int64_t n, float *out, cudaStream_t s, int cat) {
    ProfScope ps(cat, s);
    const int blocks = (int)std::min<int64_t>(152 * 4, (n * 6 + 255) / 256 + 1);
    rec_absmax_kernel<<<blocks, 256, 0, s>>>(rec, n, out);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

// tile of the tensor-core lattice sum: rows (j,l) <= 128, T0 <= 32
void tile_shape_tc(const fga_lattice &L, int T[3]) {
    if (L.n[2] == 1) {
        T[2] = 1;
        T[1] = std::min(L.n[1], 128);
    } else {
        T[2] = std::min(L.n[2], 16);
        T[1] = std::min(L.n[1], 128 / T[2]);
    }
    const int nt0 = (L.n[0] + LT_T0_MAX - 1) / LT_T0_MAX;
    T[0] = (L.n[0] + nt0 - 1) / nt0;
}

fga_status run_lattice_tc(Workspace &ws, const LatticePlan &plan, const void *rec, double k, double rw, void *u,
                          cudaStream_t s, int cat, const float *amax_in) {
    const int T0 = plan.T[0], T1 = plan.T[1], T2 = plan.T[2];
    const int TP = T0 * T1 * T2;
    if (T0 > LT_T0_MAX || T1 * T2 > LT_M || T0 + T1 + T2 > LT_TA_MAX) {
        set_error("lattice tile does not fit the tensor-core kernel");
        return FGA_ERR_UNSUPPORTED;
    }
    const int crow = 3 * T1 * T2 <= LT_M ? 1 : 0;
    const int nc_used = crow ? T0 : 3 * T0, NR = 2 * ((nc_used + 7) / 8 * 8);
    if (NR > LT_NMAX) {
        set_error("lattice tile too wide for the tensor-core kernel");
        return FGA_ERR_UNSUPPORTED;
    }
    LtSmem S;
    S.init(T0 + T1 + T2, crow && T2 == 1, NR);
    // three CTAs per SM when their tensor memory (3 x tcols <= 512) and shared memory fit
    const bool three = S.tcols <= 128 && S.bytes <= 74 * 1024;
    LtAxes X;
    for (int d = 0; d < 3; d++) {
        const int Td = plan.T[d];
        int len = plan.uniform[d] ? LT_CHUNK : 1;
        if (len > 1) {
            const double h = std::fabs(plan.dx[d]);
            len = std::min(len, 1 + (int)std::floor(recurrence_span_max(k, rw) / h));
            while (len > 1 && !recurrence_ratio_ok(k, h, (len - 1) * h, rw)) len--;
        }
        X.len[d] = len;
        X.nch[d] = (Td + X.len[d] - 1) / X.len[d];
        X.dx[d] = (float)plan.dx[d];
    }
    FGA_TRY(ws.partial.ensure(sizeof(float) * 6 * (size_t)TP * (size_t)std::max(plan.nitems, 1) + 64 +
                              sizeof(int) * (size_t)LT_CAND * (size_t)std::max(plan.nitems, 1)));
    // scratch after the partial sums: the bound of the records' amplitudes, the kept-beam lists
    char *tail = ws.partial.as<char>() + sizeof(float) * 6 * (size_t)TP * (size_t)std::max(plan.nitems, 1);
    float *amax = reinterpret_cast<float *>(tail);
    int *kept = reinterpret_cast<int *>(tail + 64);
    FGA_CUDA(cudaMemsetAsync(tail, 0, 64, s));
    if (!ws.status.p) FGA_TRY(status_reset(ws, s));
    const int cnt = prof_counting() ? 1 : 0;
    prof_add_pairs_tested(plan.pairs_tested);
    if (plan.nitems > 0) {
        if (amax_in) {
            amax = const_cast<float *>(amax_in);
        } else {
            ProfScope ps(cat, s);
            const int blocks = (int)std::min<int64_t>(152 * 4, (plan.n_rec * 6 + 255) / 256 + 1);
            rec_absmax_kernel<<<blocks, 256, 0, s>>>(static_cast<const float *>(rec), plan.n_rec, amax);
        }
        ProfScope ps(cat, s);
#define FGA_LTC(CNT, MB)                                                                                          \
    do {                                                                                                          \
        FGA_CUDA(cudaFuncSetAttribute(lattice_tc_kernel<CNT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                      S.bytes));                                                                  \
        lattice_tc_kernel<CNT, MB><<<plan.nitems, LT_THREADS, S.bytes, s>>>(                                      \
            static_cast<const float *>(rec), plan.ax[0], plan.ax[1], plan.ax[2], plan.n[0], plan.n[1], plan.n[2], \
            T0, T1, T2, plan.nt[1], plan.nt[2], plan.items, (float)k, (float)(rw * rw), amax, S, X, crow, kept,   \
            ws.partial.as<float>(), ws.status.as<int>());                                                         \
    } while (0)
        if (cnt) {
            if (three) FGA_LTC(true, 3);
            else FGA_LTC(true, 2);
        } else {
            if (three) FGA_LTC(false, 3);
            else FGA_LTC(false, 2);
        }
#undef FGA_LTC
        FGA_CUDA(cudaGetLastError());
    }
    FGA_TRY(lattice_reduce_f32(ws.partial.as<float>(), plan, u, s));
    return FGA_OK;
}

}  // namespace fga
