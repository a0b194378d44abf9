// A5-A6: cell binning of beam centres (stable LSD radix sort) and the truncated Gaussian sum of
// Eq. FGA as a gather: every CTA owns one tile of up to 32 points of one cell and one chunk of the
// beams sitting in that cell's 27 neighbours; partial sums go to scratch and a second kernel adds
// them in a fixed order (no atomics, deterministic).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "fga_beam.cuh"
#include "gather.cuh"

namespace fga {

// ---------------------------------------------------------------------------------------------
// keys
// ---------------------------------------------------------------------------------------------
template <typename TQ>
__global__ void keys_kernel(BinGrid g, const TQ *__restrict__ Q, int64_t sb, int64_t sd, int64_t n,
                            const int32_t *__restrict__ cls, int32_t *__restrict__ keys) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int cell[3];
    bool inside = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float q = (float)Q[b * sb + d * sd];
        const float t = __fmul_rn(__fsub_rn(q, g.o[d]), g.inv_h);
        const float fl = floorf(t);
        int cd;
        if (!(fl >= 0.0f)) {
            cd = 0;
            inside = false;
        } else if (fl > (float)(g.nc[d] - 1)) {
            cd = g.nc[d] - 1;
            inside = false;
        } else {
            cd = (int)fl;
        }
        cell[d] = cd;
    }
    int key = (cell[0] * g.nc[1] + cell[1]) * g.nc[2] + cell[2];
    if (!g.clamp && (!inside || (cls && (cls[b] & FL_DEAD)))) key = g.ncells;
    if (cls) key += (cls[b] & FL_CLASS_MASK) * (g.ncells + 1);
    keys[b] = key;
}

fga_status bin_centres(const BinGrid &g, const void *Q_src, int q_kind, int64_t q_stride, int64_t n,
                       const int32_t *cls_or_null, int32_t *keys, cudaStream_t s) {
    if (n == 0) return FGA_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    ProfScope ps(P_BIN, s);
    switch (q_kind) {
    case Q_F32_AOS3: keys_kernel<float><<<blocks, 256, 0, s>>>(g, (const float *)Q_src, 3, 1, n, cls_or_null, keys); break;
    case Q_F32_SOA: keys_kernel<float><<<blocks, 256, 0, s>>>(g, (const float *)Q_src, 1, q_stride, n, cls_or_null, keys); break;
    case Q_F64_SOA: keys_kernel<double><<<blocks, 256, 0, s>>>(g, (const double *)Q_src, 1, q_stride, n, cls_or_null, keys); break;
    default: set_error("bin_centres: bad source kind"); return FGA_ERR_INVALID_ARG;
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

// ---------------------------------------------------------------------------------------------
// stable LSD radix sort of (key, value) int32 pairs, 8-bit digits
// ---------------------------------------------------------------------------------------------
constexpr int RS_T = 256, RS_I = 8, RS_TILE = RS_T * RS_I;

__global__ void __launch_bounds__(RS_T) rs_hist_kernel(const int32_t *__restrict__ keys, int64_t n, int shift, int ntiles,
                                                      uint32_t *__restrict__ hist) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int r = 0; r < RS_I; r++) {
        const int64_t i = base + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) rs_scatter_kernel(const int32_t *__restrict__ kin, const int32_t *__restrict__ vin,
                                                         int64_t n, int shift, int ntiles, const uint32_t *__restrict__ off,
                                                         int32_t *__restrict__ kout, int32_t *__restrict__ vout) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[RS_T / 32][256];
    __shared__ uint32_t woff[RS_T / 32][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    run[tid] = 0;
#pragma unroll
    for (int w = 0; w < RS_T / 32; w++) wcnt[w][tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_I; r++) {
        const int64_t i = base + r * RS_T + tid;
        const bool valid = i < n;
        const int32_t key = valid ? kin[i] : 0;
        const int32_t val = valid ? vin[i] : 0;
        const int digit = valid ? ((key >> shift) & 255) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = run[tid];
#pragma unroll
            for (int w = 0; w < RS_T / 32; w++) {
                const uint32_t c = wcnt[w][tid];
                woff[w][tid] = acc;
                acc += c;
                wcnt[w][tid] = 0;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = off[(int64_t)digit * ntiles + blockIdx.x] + woff[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
    }
}

// exclusive scan of n uint32 in place: per-block scans, a one-block scan of block sums, fix-up
constexpr int SC_T = 256, SC_I = 8, SC_TILE = SC_T * SC_I;

__global__ void __launch_bounds__(SC_T) scan_block_kernel(uint32_t *__restrict__ a, int64_t n, uint32_t *__restrict__ bsum) {
    __shared__ uint32_t sh[SC_T];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_I;
    uint32_t v[SC_I], tot = 0;
#pragma unroll
    for (int j = 0; j < SC_I; j++) {
        v[j] = (base + j < n) ? a[base + j] : 0u;
        tot += v[j];
    }
    sh[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < SC_T; o <<= 1) {
        const uint32_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = sh[threadIdx.x] - tot;  // exclusive prefix of this thread
#pragma unroll
    for (int j = 0; j < SC_I; j++) {
        if (base + j < n) a[base + j] = run;
        run += v[j];
    }
    if (threadIdx.x == SC_T - 1) bsum[blockIdx.x] = sh[SC_T - 1];
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t *__restrict__ bsum, int nb) {
    // one block; nb <= 1024 * 16
    __shared__ uint32_t sh[1024];
    const int per = (nb + 1023) / 1024;
    const int beg = threadIdx.x * per;
    uint32_t tot = 0;
    for (int j = 0; j < per; j++)
        if (beg + j < nb) tot += bsum[beg + j];
    sh[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint32_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t run = sh[threadIdx.x] - tot;
    for (int j = 0; j < per; j++)
        if (beg + j < nb) {
            const uint32_t v = bsum[beg + j];
            bsum[beg + j] = run;
            run += v;
        }
}

__global__ void scan_add_kernel(uint32_t *__restrict__ a, int64_t n, const uint32_t *__restrict__ bsum) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += bsum[i / SC_TILE];
}

fga_status scan_exclusive_u32(uint32_t *a, int64_t n, cudaStream_t s);

static fga_status exclusive_scan(Workspace &ws, uint32_t *a, int64_t n, cudaStream_t s) {
    const int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    // more than 1024 x 16 block sums: the multi-level scan (it allocates its block sums)
    if (nb > 1024 * 16) return scan_exclusive_u32(a, n, s);
    FGA_TRY(ws.scan_blocks.ensure(sizeof(uint32_t) * (size_t)std::max<int64_t>(nb, 1)));
    uint32_t *bs = ws.scan_blocks.as<uint32_t>();
    {
        ProfScope ps(P_BIN, s);
        scan_block_kernel<<<(unsigned)nb, SC_T, 0, s>>>(a, n, bs);
    }
    {
        ProfScope ps(P_BIN, s);
        scan_sums_kernel<<<1, 1024, 0, s>>>(bs, (int)nb);
    }
    {
        ProfScope ps(P_BIN, s);
        scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, n, bs);
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

// the same scan for any n < 2^32 elements: the block sums of one level are scanned by the next level
fga_status scan_exclusive_u32(uint32_t *a, int64_t n, cudaStream_t s) {
    if (n <= 0) return FGA_OK;
    const int64_t nb = (n + SC_TILE - 1) / SC_TILE;
    ScopedDevBuf sums;
    FGA_TRY(sums.ensure(sizeof(uint32_t) * (size_t)nb));
    uint32_t *bs = sums.as<uint32_t>();
    {
        ProfScope ps(P_DECOMP, s);
        scan_block_kernel<<<(unsigned)nb, SC_T, 0, s>>>(a, n, bs);
    }
    FGA_CUDA(cudaGetLastError());
    if (nb <= 1024 * 16) {
        ProfScope ps(P_DECOMP, s);
        scan_sums_kernel<<<1, 1024, 0, s>>>(bs, (int)nb);
        FGA_CUDA(cudaGetLastError());
    } else {
        FGA_TRY(scan_exclusive_u32(bs, nb, s));
    }
    {
        ProfScope ps(P_DECOMP, s);
        scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, n, bs);
    }
    FGA_CUDA(cudaGetLastError());
    // the block sums are released when this scope ends
    FGA_CUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

__global__ void iota_kernel(int32_t *v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (int32_t)i;
}

fga_status radix_sort_pairs(Workspace &ws, int32_t *keys, int32_t *vals, int64_t n, int bits, int32_t **keys_out,
                            int32_t **vals_out, cudaStream_t s) {
    *keys_out = keys;
    *vals_out = vals;
    if (n <= 1) return FGA_OK;
    const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
    FGA_TRY(ws.keys_alt.ensure(sizeof(int32_t) * (size_t)n));
    FGA_TRY(ws.vals_alt.ensure(sizeof(int32_t) * (size_t)n));
    FGA_TRY(ws.hist.ensure(sizeof(uint32_t) * 256 * (size_t)ntiles));
    int32_t *ka = keys, *va = vals, *kb = ws.keys_alt.as<int32_t>(), *vb = ws.vals_alt.as<int32_t>();
    uint32_t *hist = ws.hist.as<uint32_t>();
    for (int shift = 0; shift < bits; shift += 8) {
        {
            ProfScope ps(P_BIN, s);
            rs_hist_kernel<<<ntiles, RS_T, 0, s>>>(ka, n, shift, ntiles, hist);
        }
        FGA_TRY(exclusive_scan(ws, hist, (int64_t)256 * ntiles, s));
        ProfScope ps(P_BIN, s);
        rs_scatter_kernel<<<ntiles, RS_T, 0, s>>>(ka, va, n, shift, ntiles, hist, kb, vb);
        FGA_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *keys_out = ka;
    *vals_out = va;
    return FGA_OK;
}

__global__ void cell_start_kernel(const int32_t *__restrict__ keys, int64_t n, int nbuckets, int32_t *__restrict__ start) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    const int prev = i == 0 ? -1 : keys[i - 1];
    const int cur = i == n ? nbuckets : keys[i];
    for (int c = prev + 1; c <= cur; c++) start[c] = (int32_t)i;
}

fga_status cell_starts(const int32_t *sorted_keys, int64_t n, int nbuckets, int32_t *cell_start, cudaStream_t s) {
    ProfScope ps(P_BIN, s);
    cell_start_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(sorted_keys, n, nbuckets, cell_start);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

fga_status sort_keys_to_perm(Workspace &ws, int32_t *keys, int64_t n, int nbuckets, int32_t **perm_out,
                             int32_t *cell_start, cudaStream_t s) {
    FGA_TRY(ws.vals.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
    int32_t *vals = ws.vals.as<int32_t>();
    ProfScope ps(P_BIN, s);
    if (n > 0) iota_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(vals, n);
    int bits = 0;
    while ((1ll << bits) < (long long)nbuckets) bits++;
    bits = std::max(8, (bits + 7) / 8 * 8);
    int32_t *ks, *vs;
    FGA_TRY(radix_sort_pairs(ws, keys, vals, n, bits, &ks, &vs, s));
    FGA_TRY(cell_starts(ks, n, nbuckets, cell_start, s));
    *perm_out = vs;
    return FGA_OK;
}

// ---------------------------------------------------------------------------------------------
// permutation of the beam state (sorted by cell, once per window of steps)
// ---------------------------------------------------------------------------------------------
template <typename R>
__global__ void permute_kernel(const R *__restrict__ src, R *__restrict__ dst, const int32_t *__restrict__ fsrc,
                               int32_t *__restrict__ fdst, const int32_t *__restrict__ isrc, int32_t *__restrict__ idst,
                               const int32_t *__restrict__ perm, int64_t n, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t j = perm[i];
#pragma unroll 2
    for (int f = 0; f < NFS; f++) dst[(int64_t)f * cap + i] = src[(int64_t)f * cap + j];
    fdst[i] = fsrc[j];
    idst[i] = isrc[j];
}

fga_status permute_beams(fga_beams *b, const int32_t *perm, cudaStream_t s) {
    const size_t rb = b->precision == FGA_PREC_FP64 ? 8 : 4;
    FGA_TRY(b->state_alt.ensure(rb * NFS * b->cap));
    FGA_TRY(b->flags_alt.ensure(4 * b->cap));
    FGA_TRY(b->id_alt.ensure(4 * b->cap));
    const unsigned blocks = (unsigned)((b->nb + 255) / 256);
    if (b->nb > 0) {
        ProfScope ps(P_BIN, s);
        if (rb == 8)
            permute_kernel<double><<<blocks, 256, 0, s>>>(b->state.as<double>(), b->state_alt.as<double>(),
                                                          b->flags.as<int32_t>(), b->flags_alt.as<int32_t>(),
                                                          b->id.as<int32_t>(), b->id_alt.as<int32_t>(), perm, b->nb, b->cap);
        else
            permute_kernel<float><<<blocks, 256, 0, s>>>(b->state.as<float>(), b->state_alt.as<float>(),
                                                         b->flags.as<int32_t>(), b->flags_alt.as<int32_t>(),
                                                         b->id.as<int32_t>(), b->id_alt.as<int32_t>(), perm, b->nb, b->cap);
        FGA_CUDA(cudaGetLastError());
    }
    std::swap(b->state, b->state_alt);
    std::swap(b->flags, b->flags_alt);
    std::swap(b->id, b->id_alt);
    return FGA_OK;
}

// ---------------------------------------------------------------------------------------------
// Gaussian sum
// ---------------------------------------------------------------------------------------------
BinGrid make_grid(const double *pts, int64_t n, double reach) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) {
            lo[d] = std::min(lo[d], pts[3 * i + d]);
            hi[d] = std::max(hi[d], pts[3 * i + d]);
        }
    if (n == 0)
        for (int d = 0; d < 3; d++) lo[d] = hi[d] = 0.0;
    BinGrid g;
    const double h = reach * 1.001;  // slack for FP32 key rounding
    g.inv_h = (float)(1.0 / h);
    g.ncells = 1;
    for (int d = 0; d < 3; d++) {
        g.o[d] = (float)(lo[d] - reach * 1.0005);
        const double ext = hi[d] + reach * 1.0005 - (double)g.o[d];
        g.nc[d] = std::max(1, (int)std::ceil(ext * (double)g.inv_h));
        g.ncells *= g.nc[d];
    }
    g.clamp = false;
    return g;
}

// (beam, point) pairs that fell inside the window, counted when profiling is on
static __device__ unsigned long long g_pairs_in_window;

int64_t read_pair_counter(bool reset) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_pairs_in_window, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_pairs_in_window, &z, sizeof z);
    }
    return (int64_t)v;
}

template <typename R>
__global__ void __launch_bounds__(128) gather_kernel(const R *__restrict__ rec, const double *__restrict__ pts,
                                                    const int32_t *__restrict__ tile_pts, const int4 *__restrict__ items,
                                                    R k, R rw2, R *__restrict__ partial, int count_pairs) {
    __shared__ R red[4][32][6];
    __shared__ unsigned npairs;
    if (threadIdx.x == 0) npairs = 0;
    unsigned mine = 0;
    const int4 it = items[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pi = tile_pts[it.x * 32 + lane];
    R x0, x1, x2;
    if (pi >= 0) {
        x0 = (R)pts[3 * (int64_t)pi];
        x1 = (R)pts[3 * (int64_t)pi + 1];
        x2 = (R)pts[3 * (int64_t)pi + 2];
    } else {
        x0 = x1 = x2 = R(1e30);
    }
    const int64_t len = (int64_t)it.z - it.y;
    const int64_t b0 = it.y + (len * warp) / 4, b1 = it.y + (len * (warp + 1)) / 4;
    R acc[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const R hk = R(-0.5) * k;
    for (int64_t b = b0; b < b1; b++) {
        const R *r = rec + b * REC;
        R q[REC];
        if (sizeof(R) == 4) {
            const float4 *r4 = reinterpret_cast<const float4 *>(r);
            const float4 u0 = __ldg(r4), u1 = __ldg(r4 + 1), u2 = __ldg(r4 + 2);
            const float t[12] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
#pragma unroll
            for (int j = 0; j < REC; j++) q[j] = (R)t[j];
        } else {
            const double2 *r2 = reinterpret_cast<const double2 *>(r);
#pragma unroll
            for (int j = 0; j < 6; j++) {
                const double2 v = __ldg(r2 + j);
                q[2 * j] = (R)v.x;
                q[2 * j + 1] = (R)v.y;
            }
        }
        const R d0 = x0 - q[0], d1 = x1 - q[1], d2 = x2 - q[2];
        const R r2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (r2 <= rw2) {
            mine++;
            const R ph = k * (q[3] * d0 + q[4] * d1 + q[5] * d2);
            R er, ei;
            gauss_phase_exp<R>(ph, hk * r2, &er, &ei);
#pragma unroll
            for (int d = 0; d < 3; d++) cmac<R>(acc[2 * d], acc[2 * d + 1], q[6 + 2 * d], q[7 + 2 * d], er, ei);
        }
    }
#pragma unroll
    for (int j = 0; j < 6; j++) red[warp][lane][j] = acc[j];
    if (count_pairs) atomicAdd(&npairs, mine);
    __syncthreads();
    if (count_pairs && threadIdx.x == 0) atomicAdd(&g_pairs_in_window, (unsigned long long)npairs);
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const R v = (red[0][lane][j] + red[1][lane][j]) + (red[2][lane][j] + red[3][lane][j]);
            partial[((int64_t)blockIdx.x * 32 + lane) * 6 + j] = v;
        }
    }
}

template <typename R>
__global__ void reduce_kernel(const R *__restrict__ partial, const int32_t *__restrict__ tile_pts,
                              const int32_t *__restrict__ item_start, int ntiles, R *__restrict__ u) {
    const int t = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const int pi = tile_pts[t * 32 + lane];
    if (pi < 0) return;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = item_start[t]; i < item_start[t + 1]; i++)
#pragma unroll
        for (int j = 0; j < 6; j++) acc[j] += (double)partial[((int64_t)i * 32 + lane) * 6 + j];
#pragma unroll
    for (int j = 0; j < 6; j++) u[(int64_t)pi * 6 + j] = (R)acc[j];
}

fga_status build_sum_plan(Workspace &ws, const BinGrid &g, const int32_t *cell_start_dev, int nclasses,
                          const double *pts_host, int64_t npts, cudaStream_t s, SumPlan &plan) {
    plan.ntiles = 0;
    plan.nitems = 0;
    if (npts == 0) return FGA_OK;
    const int nbk = nclasses * (g.ncells + 1);
    FGA_TRY(ws.h_cell_start.ensure(sizeof(int32_t) * (size_t)(nbk + 1)));
    int32_t *cs = ws.h_cell_start.as<int32_t>();
    FGA_CUDA(cudaMemcpyAsync(cs, cell_start_dev, sizeof(int32_t) * (size_t)(nbk + 1), cudaMemcpyDeviceToHost, s));
    // points -> cells (host, FP64; the cell size carries slack for the FP32 beam keys)
    std::vector<int32_t> pcell((size_t)npts);
    for (int64_t i = 0; i < npts; i++) {
        int c[3];
        for (int d = 0; d < 3; d++) {
            const double t = (pts_host[3 * i + d] - (double)g.o[d]) * (double)g.inv_h;
            int cd = (int)std::floor(t);
            cd = std::min(std::max(cd, 0), g.nc[d] - 1);
            c[d] = cd;
        }
        pcell[(size_t)i] = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
    }
    std::vector<int32_t> order((size_t)npts);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return pcell[a] < pcell[b]; });
    std::vector<int32_t> tiles;  // 32 entries per tile
    std::vector<int32_t> tile_cell;
    for (int64_t i = 0; i < npts;) {
        const int cell = pcell[(size_t)order[(size_t)i]];
        int64_t j = i;
        while (j < npts && pcell[(size_t)order[(size_t)j]] == cell) j++;
        for (int64_t t0 = i; t0 < j; t0 += 32) {
            for (int l = 0; l < 32; l++) tiles.push_back(t0 + l < j ? order[(size_t)(t0 + l)] : -1);
            tile_cell.push_back(cell);
        }
        i = j;
    }
    const int ntiles = (int)tile_cell.size();
    FGA_CUDA(cudaStreamSynchronize(s));  // cell_start on the host
    plan.n_rec = 0;
    for (int cl = 0; cl < 4; cl++) {
        plan.n_in[cl] = 0;
        plan.rec_off[cl] = plan.n_rec;
        if (cl < nclasses) {
            const int cb = cl * (g.ncells + 1);
            plan.n_in[cl] = cs[cb + g.ncells] - cs[cb];
            plan.beg[cl] = cs[cb];
        }
        plan.n_rec += plan.n_in[cl];
    }
    // candidate ranges per tile: (c0 +- 1, c1 +- 1) x contiguous c2 - 1 .. c2 + 1, per class
    struct Rg {
        int tile, b, e;
    };
    std::vector<Rg> ranges;
    int64_t total = 0;
    for (int t = 0; t < ntiles; t++) {
        const int cell = tile_cell[(size_t)t];
        const int c2 = cell % g.nc[2], c1 = (cell / g.nc[2]) % g.nc[1], c0 = cell / (g.nc[2] * g.nc[1]);
        const int lo2 = std::max(c2 - 1, 0), hi2 = std::min(c2 + 1, g.nc[2] - 1);
        for (int cl = 0; cl < nclasses; cl++) {
            const int cb = cl * (g.ncells + 1);
            for (int a0 = std::max(c0 - 1, 0); a0 <= std::min(c0 + 1, g.nc[0] - 1); a0++)
                for (int a1 = std::max(c1 - 1, 0); a1 <= std::min(c1 + 1, g.nc[1] - 1); a1++) {
                    const int id0 = (a0 * g.nc[1] + a1) * g.nc[2];
                    // sorted positions -> compact record indices of class cl
                    const int64_t shift = plan.rec_off[cl] - cs[cb];
                    const int bb = (int)(cs[cb + id0 + lo2] + shift), ee = (int)(cs[cb + id0 + hi2 + 1] + shift);
                    if (ee > bb) {
                        ranges.push_back({t, bb, ee});
                        total += ee - bb;
                    }
                }
        }
    }
    // chunk size: aim at >= ~4096 work items so that every SM has several CTAs
    int64_t B = std::max<int64_t>(512, (total + 4095) / 4096);
    B = (B + 127) / 128 * 128;
    std::vector<int32_t> item_start((size_t)ntiles + 1, 0);
    std::vector<int4> items;
    size_t ri = 0;
    for (int t = 0; t < ntiles; t++) {
        item_start[(size_t)t] = (int32_t)items.size();
        while (ri < ranges.size() && ranges[ri].tile == t) {
            for (int64_t b = ranges[ri].b; b < ranges[ri].e; b += B)
                items.push_back(make_int4(t, (int)b, (int)std::min<int64_t>(b + B, ranges[ri].e), 0));
            ri++;
        }
    }
    item_start[(size_t)ntiles] = (int32_t)items.size();
    plan.ntiles = ntiles;
    plan.nitems = (int)items.size();
    const size_t tb = sizeof(int32_t) * tiles.size(), ib = sizeof(int4) * items.size(),
                 sb = sizeof(int32_t) * item_start.size();
    FGA_TRY(ws.tiles.ensure(tb + sb));
    FGA_TRY(ws.items.ensure(std::max<size_t>(ib, 16)));
    FGA_TRY(ws.h_tiles.ensure(tb + sb));
    FGA_TRY(ws.h_items.ensure(std::max<size_t>(ib, 16)));
    std::memcpy(ws.h_tiles.p, tiles.data(), tb);
    std::memcpy(static_cast<char *>(ws.h_tiles.p) + tb, item_start.data(), sb);
    if (ib) std::memcpy(ws.h_items.p, items.data(), ib);
    FGA_CUDA(cudaMemcpyAsync(ws.tiles.p, ws.h_tiles.p, tb + sb, cudaMemcpyHostToDevice, s));
    if (ib) FGA_CUDA(cudaMemcpyAsync(ws.items.p, ws.h_items.p, ib, cudaMemcpyHostToDevice, s));
    plan.tile_pts = ws.tiles.as<int32_t>();
    plan.item_start = reinterpret_cast<int32_t *>(static_cast<char *>(ws.tiles.p) + tb);
    plan.items = ws.items.as<int4>();
    plan.pairs_tested = total * 32;
    return FGA_OK;
}

const int32_t *plan_host_cell_start(const Workspace &ws) { return ws.h_cell_start.as<int32_t>(); }

fga_status run_sum(Workspace &ws, const SumPlan &plan, int precision, const void *rec_sorted, const double *pts_dev,
                   double k, double rw, void *u_out, cudaStream_t s, int cat) {
    if (plan.ntiles == 0) return FGA_OK;
    const size_t rb = precision == FGA_PREC_FP64 ? 8 : 4;
    FGA_TRY(ws.partial.ensure(rb * 32 * 6 * (size_t)std::max(plan.nitems, 1)));
    const int cnt = prof_counting() ? 1 : 0;
    prof_add_pairs_tested(plan.pairs_tested);
    if (plan.nitems > 0) {
        ProfScope ps(cat, s);
        if (rb == 8)
            gather_kernel<double><<<plan.nitems, 128, 0, s>>>((const double *)rec_sorted, pts_dev, plan.tile_pts,
                                                              plan.items, k, rw * rw, ws.partial.as<double>(), cnt);
        else
            gather_kernel<float><<<plan.nitems, 128, 0, s>>>((const float *)rec_sorted, pts_dev, plan.tile_pts,
                                                             plan.items, (float)k, (float)(rw * rw), ws.partial.as<float>(),
                                                             cnt);
        FGA_CUDA(cudaGetLastError());
    }
    const int tpb = 4;  // tiles per 128-thread block
    const unsigned blocks = (unsigned)((plan.ntiles + tpb - 1) / tpb);
    ProfScope ps(P_REDUCE, s);
    if (rb == 8)
        reduce_kernel<double><<<blocks, 32 * tpb, 0, s>>>(ws.partial.as<double>(), plan.tile_pts, plan.item_start,
                                                          plan.ntiles, (double *)u_out);
    else
        reduce_kernel<float><<<blocks, 32 * tpb, 0, s>>>(ws.partial.as<float>(), plan.tile_pts, plan.item_start,
                                                         plan.ntiles, (float *)u_out);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

}  // namespace fga
