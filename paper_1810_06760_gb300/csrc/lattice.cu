// A6 on tensor lattices of points (snapshot grids, receiver arrays): the truncated Gaussian sum of
// Eq. FGA, using that exp(i k P.(x-Q) - k|x-Q|^2/2) = prod_d E_d(x_d) with
// E_d(x) = exp(i k P_d (x - Q_d) - k (x - Q_d)^2 / 2).  A CTA owns a box ("tile") of the lattice
// and a chunk of the cell-binned beams near it; per beam it forms the 1-D factors of the tile's
// coordinates once (T0 + T1 + T2 complex exponentials) and every point of the tile then costs one
// complex product per component -- no transcendental per point.  The window |x - Q| <= rw is
// still tested per point, from per-axis squared distances.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fga_beam.cuh"
#include "gather.cuh"

namespace fga {

// (beam, point) pairs inside the window, counted when profiling is on
static __device__ unsigned long long g_lattice_pairs;

int64_t read_lattice_pair_counter(bool reset) {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_lattice_pairs, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_lattice_pairs, &z, sizeof z);
    }
    return (int64_t)v;
}

// Shared-memory layout of one batch of at most NB kept beams (runtime tile T0 x T1 x T2):
//   ae0[b][i]  = (A_c E0(x_i) for c = 0..2 as re/im, (x_i - Q_0)^2, 0)              8 reals
//   ed12[b][jl] = (E1(x_j) E2(x_l) re/im, (x_j - Q_1)^2 + (x_l - Q_2)^2, 0)         4 reals
// so that a point reads its beam terms with three 16-byte (FP32) loads.
struct LatSmem {
    int NB, T0, T1, T2, T12, TP, B0, B1, B2, nblk0, nblk1, nblk2;
    size_t rec, mask, ae0, ed12, e1, e2, x, bytes;
    template <typename R> __host__ __device__ void init(int nb, int t0, int t1, int t2) {
        NB = nb;
        T0 = t0;
        T1 = t1;
        T2 = t2;
        T12 = t1 * t2;
        TP = t0 * T12;
        // warp blocks of 32 points, compact in the lattice: 4 x 8 x 1 on planes, 2 x 4 x 4 in volumes
        if (T2 == 1) {
            B0 = 4;
            B1 = 8;
            B2 = 1;
        } else {
            B0 = 2;
            B1 = 4;
            B2 = 4;
        }
        nblk0 = (T0 + B0 - 1) / B0;
        nblk1 = (T1 + B1 - 1) / B1;
        nblk2 = (T2 + B2 - 1) / B2;
        size_t o = 0;
        auto take = [&](size_t n) {
            const size_t r = o;
            o += (n * sizeof(R) + 15) / 16 * 16;
            return r;
        };
        rec = take((size_t)NB * REC);
        mask = take((size_t)NB * (sizeof(unsigned) + sizeof(R) - 1) / sizeof(R));
        ae0 = take((size_t)NB * T0 * 8);
        ed12 = take((size_t)NB * T12 * 4);
        e1 = take((size_t)NB * T1 * 4);
        e2 = take((size_t)NB * T2 * 4);
        x = take((size_t)(T0 + T1 + T2));
        bytes = o;
    }
    __host__ __device__ int nblocks() const { return nblk0 * nblk1 * nblk2; }
};

template <typename R> struct V4;
template <> struct V4<float> {
    using T = float4;
};
template <> struct V4<double> {
    using T = double4;
};

// One CTA = one (tile, chunk of candidate beams).  Per batch: the first NB threads hold candidate
// records (loaded one batch ahead) and keep those within rw of the tile's box; warps form the kept
// beams' 1-D factors and which warp blocks each beam reaches; then every warp adds the batch to its
// blocks of 32 points, skipping (warp-uniformly) blocks the beam cannot reach.
template <typename R, int PTS, bool COUNT>
__global__ void __launch_bounds__(256) lattice_gather_kernel(const R *__restrict__ rec, const double *__restrict__ ax0,
                                                            const double *__restrict__ ax1, const double *__restrict__ ax2,
                                                            int n0, int n1, int n2, LatSmem L, int nt1, int nt2,
                                                            const int4 *__restrict__ items, R k, R rw2,
                                                            R *__restrict__ partial) {
    using R4 = typename V4<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    R *s_rec = reinterpret_cast<R *>(smem + L.rec);
    R4 *s_ae0 = reinterpret_cast<R4 *>(smem + L.ae0);    // [NB][T0][2]
    R4 *s_ed12 = reinterpret_cast<R4 *>(smem + L.ed12);  // [NB][T12]
    R4 *s_e1 = reinterpret_cast<R4 *>(smem + L.e1);       // [NB][T1]: re, im, d^2, -
    R4 *s_e2 = reinterpret_cast<R4 *>(smem + L.e2);       // [NB][T2]
    R *s_x = reinterpret_cast<R *>(smem + L.x);
    unsigned *s_mask = reinterpret_cast<unsigned *>(smem + L.mask);  // [NB]: warp blocks within rw
    __shared__ int s_wcnt[2];
    __shared__ unsigned s_pairs;
    const int T0 = L.T0, T1 = L.T1, T2 = L.T2, T12 = L.T12, NB = L.NB, TA = T0 + T1 + T2;

    const int4 it = items[blockIdx.x];
    const int t = it.x;
    const int tt0 = t / (nt1 * nt2), tt1 = (t / nt2) % nt1, tt2 = t % nt2;
    const int i0 = tt0 * T0, j0 = tt1 * T1, l0 = tt2 * T2;
    const int e0 = min(T0, n0 - i0), e1 = min(T1, n1 - j0), e2 = min(T2, n2 - l0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int a = tid; a < TA; a += 256) {
        R v;
        if (a < T0) v = (R)ax0[i0 + min(a, e0 - 1)];
        else if (a < T0 + T1) v = (R)ax1[j0 + min(a - T0, e1 - 1)];
        else v = (R)ax2[l0 + min(a - T0 - T1, e2 - 1)];
        s_x[a] = v;
    }
    if (tid == 0) s_pairs = 0;
    __syncthreads();
    const R lo0 = s_x[0], hi0 = s_x[T0 - 1], lo1 = s_x[T0], hi1 = s_x[T0 + T1 - 1];
    const R lo2 = s_x[T0 + T1], hi2 = s_x[TA - 1];

    // this thread's points: lane (di, dj, dl) of warp blocks warp + 8 q; offsets into the factors
    int o12[PTS], o0[PTS];
    bool pin[PTS];
    unsigned pval[PTS];
    {
        const int dl = lane % L.B2, dj = (lane / L.B2) % L.B1, di = lane / (L.B2 * L.B1);
#pragma unroll
        for (int q = 0; q < PTS; q++) {
            const int blk = warp + 8 * q;
            const int b2 = blk % L.nblk2, b1 = (blk / L.nblk2) % L.nblk1, b0 = blk / (L.nblk2 * L.nblk1);
            const int i = b0 * L.B0 + di, j = b1 * L.B1 + dj, l = b2 * L.B2 + dl;
            pin[q] = blk < L.nblocks() && i < T0 && j < T1 && l < T2;
            o12[q] = pin[q] ? j * T2 + l : 0;
            o0[q] = pin[q] ? 2 * i : 0;
            pval[q] = (pin[q] && i < e0 && j < e1 && l < e2) ? 1u : 0u;
        }
    }
    // warp-block boxes of this lane's block (for the reach masks)
    const int nblk = L.nblocks();
    R blo[3] = {R(0), R(0), R(0)}, bhi[3] = {R(0), R(0), R(0)};
    if (lane < nblk) {
        const int b2 = lane % L.nblk2, b1 = (lane / L.nblk2) % L.nblk1, b0 = lane / (L.nblk2 * L.nblk1);
        const int ia = b0 * L.B0, ja = b1 * L.B1, la = b2 * L.B2;
        blo[0] = s_x[ia];
        bhi[0] = s_x[min(ia + L.B0, T0) - 1];
        blo[1] = s_x[T0 + ja];
        bhi[1] = s_x[T0 + min(ja + L.B1, T1) - 1];
        blo[2] = s_x[T0 + T1 + la];
        bhi[2] = s_x[T0 + T1 + min(la + L.B2, T2) - 1];
    }
    R acc[PTS][6];
#pragma unroll
    for (int q = 0; q < PTS; q++)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[q][c] = R(0);
    unsigned mine = 0;
    const R hk = R(-0.5) * k;

    R r[REC];
    auto load = [&](int64_t bbase) {
        const int64_t b = bbase + tid;
        if (tid < NB && b < it.z) {
#pragma unroll
            for (int q = 0; q < REC; q++) r[q] = rec[b * REC + q];
        }
    };
    load(it.y);
    for (int64_t base = it.y; base < it.z; base += NB) {
        // 1. candidates -> kept beams (order preserved)
        bool keep = false;
        if (tid < NB && base + tid < it.z) {
            const R g0 = fmax(fmax(lo0 - r[0], r[0] - hi0), R(0));
            const R g1 = fmax(fmax(lo1 - r[1], r[1] - hi1), R(0));
            const R g2 = fmax(fmax(lo2 - r[2], r[2] - hi2), R(0));
            keep = g0 * g0 + g1 * g1 + g2 * g2 <= rw2;
        }
        unsigned m = 0;
        if (warp < 2) {
            m = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_wcnt[warp] = __popc(m);
        }
        __syncthreads();
        const int nb = s_wcnt[0] + (NB > 32 ? s_wcnt[1] : 0);
        if (keep) {
            const int slot = (warp ? s_wcnt[0] : 0) + __popc(m & ((1u << lane) - 1u));
#pragma unroll
            for (int q = 0; q < REC; q++) s_rec[slot * REC + q] = r[q];
        }
        __syncthreads();
        load(base + NB);  // next batch, in flight during the work below
        if (nb == 0) continue;
        // 2a. reach masks (a warp per kept beam, lane = warp block)
        for (int b = warp; b < nb; b += 8) {
            const R *rb = s_rec + b * REC;
            const R g0 = fmax(fmax(blo[0] - rb[0], rb[0] - bhi[0]), R(0));
            const R g1 = fmax(fmax(blo[1] - rb[1], rb[1] - bhi[1]), R(0));
            const R g2 = fmax(fmax(blo[2] - rb[2], rb[2] - bhi[2]), R(0));
            const unsigned bm = __ballot_sync(0xffffffffu, lane < nblk && g0 * g0 + g1 * g1 + g2 * g2 <= rw2);
            if (lane == 0) s_mask[b] = bm;
        }
        // 2b. 1-D factors: every (beam, tile coordinate) pair is one task, spread over all threads
        // (b = floor((e + 1/2) / TA) is exact in FP32 for these small integers)
        {
            const float inv_ta = 1.0f / (float)TA;
            for (int e = tid; e < nb * TA; e += 256) {
                const int b = (int)(((float)e + 0.5f) * inv_ta), a = e - b * TA;
                const R *rb = s_rec + b * REC;
                const int d = a < T0 ? 0 : (a < T0 + T1 ? 1 : 2);
                const R dx = s_x[a] - rb[d];
                R er, ei;
                gauss_phase_exp<R>(k * rb[3 + d] * dx, hk * dx * dx, &er, &ei);
                if (d == 0) {
                    R o[6];
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        const R ar = rb[6 + 2 * c], ai = rb[7 + 2 * c];
                        o[2 * c] = ar * er - ai * ei;
                        o[2 * c + 1] = ar * ei + ai * er;
                    }
                    R4 *dst = s_ae0 + (b * T0 + a) * 2;
                    dst[0] = R4{o[0], o[1], o[2], o[3]};
                    dst[1] = R4{o[4], o[5], dx * dx, R(0)};
                } else if (d == 1) {
                    s_e1[b * T1 + (a - T0)] = R4{er, ei, dx * dx, R(0)};
                } else {
                    s_e2[b * T2 + (a - T0 - T1)] = R4{er, ei, dx * dx, R(0)};
                }
            }
        }
        __syncthreads();
        {
            const float inv_t12 = 1.0f / (float)T12, inv_t2 = 1.0f / (float)T2;
            for (int e = tid; e < nb * T12; e += 256) {
                const int b = (int)(((float)e + 0.5f) * inv_t12), jl = e - b * T12;
                const int j = (int)(((float)jl + 0.5f) * inv_t2), l = jl - j * T2;
                const R4 u = s_e1[b * T1 + j], v = s_e2[b * T2 + l];
                s_ed12[e] = R4{u.x * v.x - u.y * v.y, u.x * v.y + u.y * v.x, u.z + v.z, R(0)};
            }
        }
        __syncthreads();
        // 3. the batch's contribution to this thread's points
        for (int b = 0; b < nb; b++) {
            const unsigned bm = s_mask[b];
            const R4 *ed = s_ed12 + b * T12;
            const R4 *ae = s_ae0 + b * 2 * T0;
#pragma unroll
            for (int q = 0; q < PTS; q++) {
                if ((bm >> (warp + 8 * q)) & 1u) {
                    const R4 e = ed[o12[q]];
                    const R4 a0 = ae[o0[q]], a1 = ae[o0[q] + 1];
                    if (pin[q] && a1.z + e.z <= rw2) {
                        if (COUNT) mine += pval[q];
                        cmac<R>(acc[q][0], acc[q][1], a0.x, a0.y, e.x, e.y);
                        cmac<R>(acc[q][2], acc[q][3], a0.z, a0.w, e.x, e.y);
                        cmac<R>(acc[q][4], acc[q][5], a1.x, a1.y, e.x, e.y);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PTS; q++) {
        if (pin[q]) {
            R *dst = partial + ((int64_t)blockIdx.x * L.TP + (o0[q] / 2) * T12 + o12[q]) * 6;
#pragma unroll
            for (int c = 0; c < 6; c++) dst[c] = acc[q][c];
        }
    }
    if (COUNT) {
        atomicAdd(&s_pairs, mine);
        __syncthreads();
        if (tid == 0) atomicAdd(&g_lattice_pairs, (unsigned long long)s_pairs);
    }
}

// u at every lattice point: a warp per point, lanes striding over the tile's items, then a fixed
// shuffle tree (deterministic for a given work split)
template <typename R>
__global__ void lattice_reduce_kernel(const R *__restrict__ partial, const int32_t *__restrict__ item_start, int n0,
                                      int n1, int n2, int T0, int T1, int T2, int nt1, int nt2, R *__restrict__ u) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)n0 * n1 * n2;
    if (g >= total) return;
    const int l = (int)(g % n2), j = (int)((g / n2) % n1), i = (int)(g / ((int64_t)n1 * n2));
    const int t = ((i / T0) * nt1 + j / T1) * nt2 + l / T2;
    const int p = ((i % T0) * T1 + j % T1) * T2 + l % T2;
    const int TP = T0 * T1 * T2;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int it = item_start[t] + lane; it < item_start[t + 1]; it += 32)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += (double)partial[((int64_t)it * TP + p) * 6 + c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane < 6) {
        double v = acc[0];
#pragma unroll
        for (int c = 1; c < 6; c++)
            if (lane == c) v = acc[c];
        u[g * 6 + lane] = (R)v;
    }
}

// tile shape: at most 1024 points and 64 per axis; axis 2 first (up to 16), then 1, then 0
static void tile_shape(const fga_lattice &L, int T[3]) {
    T[2] = std::min(L.n[2], 16);
    T[1] = std::min(L.n[1], std::max(1, std::min(64, 1024 / (T[2] * std::min(L.n[0], 8)))));
    T[0] = std::min(L.n[0], std::max(1, std::min(64, 1024 / (T[1] * T[2]))));
    // at most 32 warp blocks (4 per warp of a 256-thread CTA)
    const int B0 = T[2] == 1 ? 4 : 2, B1 = T[2] == 1 ? 8 : 4, B2 = T[2] == 1 ? 1 : 4;
    auto nblk = [&]() { return ((T[0] + B0 - 1) / B0) * ((T[1] + B1 - 1) / B1) * ((T[2] + B2 - 1) / B2); };
    while (nblk() > 32) {
        if (T[0] > B0) T[0] -= B0;
        else if (T[1] > B1) T[1] -= B1;
        else T[2] -= B2;
    }
}

double recurrence_span_max(double k, double rw) {
    const double sk = std::sqrt(k);
    return std::max((std::sqrt(174.0) - std::sqrt(28.0)) / sk, std::sqrt(174.0) / sk - rw);
}
bool recurrence_ratio_ok(double k, double step, double span, double rw) {
    return k * std::fabs(step) * (span + rw + std::fabs(step)) <= 87.0;
}

// the plane kernel's runs: axis 1 in two halves of ceil(T1/2) points (step h1), axis 0 in the two
// parities of ceil(T0/2) points (step 2 h0); cap T so every run stays within the recurrence limits
static void cap_plane_tile(const LatticePlan &plan, double k, double rw, int T[3]) {
    const double smax = recurrence_span_max(k, rw);
    for (int d = 0; d < 2; d++) {
        if (T[d] <= 2 || !plan.uniform[d]) continue;
        const double step = (d == 0 ? 2.0 : 1.0) * std::fabs(plan.dx[d]);
        int J = 1 + (int)std::floor(smax / step);
        while (J > 1 && !recurrence_ratio_ok(k, step, (J - 1) * step, rw)) J--;
        T[d] = std::min(T[d], 2 * J);
    }
}

fga_status build_lattice_plan(Workspace &ws, const BinGrid &g, const int32_t *cell_start_dev, const fga_lattice &L,
                              cudaStream_t s, LatticePlan &plan, bool tc, double k, double rw) {
    // axes with uniform spacing (the tensor-core kernels form their 1-D factors by recurrence there)
    for (int d = 0; d < 3; d++) {
        const double *a = L.axis[d];
        const int n = L.n[d];
        bool uni = n >= 2;
        const double step = n >= 2 ? (a[n - 1] - a[0]) / (n - 1) : 0.0;
        const double scale = std::max(std::fabs(a[0]), std::fabs(a[n - 1])) + std::fabs(step) * n;
        for (int i = 0; uni && i < n; i++) uni = std::fabs(a[i] - (a[0] + i * step)) <= 1e-12 * scale;
        plan.uniform[d] = uni && step != 0.0;
        plan.dx[d] = step;
        plan.x_first[d] = a[0];
    }
    const bool plane = tc && L.n[2] == 1 && (plan.uniform[0] || L.n[0] == 1) && (plan.uniform[1] || L.n[1] == 1);
    int T[3];
    if (plane) {
        tile_shape_plane(L, T);
        cap_plane_tile(plan, k, rw, T);
    } else if (tc)
        tile_shape_tc(L, T);
    else
        tile_shape(L, T);
    plan.T[0] = T[0];
    plan.T[1] = T[1];
    plan.T[2] = T[2];
    for (int d = 0; d < 3; d++) {
        plan.n[d] = L.n[d];
        plan.nt[d] = (L.n[d] + T[d] - 1) / T[d];
    }
    const int ntiles = plan.nt[0] * plan.nt[1] * plan.nt[2];
    const int nbk = 4 * (g.ncells + 1);
    FGA_TRY(ws.h_cell_start.ensure(sizeof(int32_t) * (size_t)(nbk + 1)));
    int32_t *cs = ws.h_cell_start.as<int32_t>();
    FGA_CUDA(cudaMemcpyAsync(cs, cell_start_dev, sizeof(int32_t) * (size_t)(nbk + 1), cudaMemcpyDeviceToHost, s));
    FGA_CUDA(cudaStreamSynchronize(s));
    plan.n_rec = 0;
    for (int cl = 0; cl < 4; cl++) {
        const int cb = cl * (g.ncells + 1);
        plan.n_in[cl] = cs[cb + g.ncells] - cs[cb];
        plan.beg[cl] = cs[cb];
        plan.rec_off[cl] = plan.n_rec;
        plan.n_rec += plan.n_in[cl];
    }
    auto cell_of = [&](int d, double x) {
        int c = (int)std::floor((x - (double)g.o[d]) * (double)g.inv_h);
        return std::min(std::max(c, 0), g.nc[d] - 1);
    };
    struct Rg {
        int tile, b, e;
    };
    std::vector<Rg> ranges;
    int64_t total = 0;
    for (int t = 0; t < ntiles; t++) {
        const int tt[3] = {t / (plan.nt[1] * plan.nt[2]), (t / plan.nt[2]) % plan.nt[1], t % plan.nt[2]};
        int clo[3], chi[3];
        for (int d = 0; d < 3; d++) {
            const int a0 = tt[d] * T[d], a1 = std::min(L.n[d], a0 + T[d]) - 1;
            clo[d] = std::max(cell_of(d, L.axis[d][a0]) - 1, 0);
            chi[d] = std::min(cell_of(d, L.axis[d][a1]) + 1, g.nc[d] - 1);
        }
        for (int cl = 0; cl < 4; cl++) {
            const int cb = cl * (g.ncells + 1);
            const int64_t shift = plan.rec_off[cl] - cs[cb];
            for (int a0 = clo[0]; a0 <= chi[0]; a0++)
                for (int a1 = clo[1]; a1 <= chi[1]; a1++) {
                    const int id0 = (a0 * g.nc[1] + a1) * g.nc[2];
                    const int bb = (int)(cs[cb + id0 + clo[2]] + shift), ee = (int)(cs[cb + id0 + chi[2] + 1] + shift);
                    if (ee > bb) {
                        ranges.push_back({t, bb, ee});
                        total += ee - bb;
                    }
                }
        }
    }
    // beams per work item: the tensor-core kernels amortise their set-up over longer ranges (the plane
    // kernel runs one persistent CTA per SM over about three items each)
    int64_t B = plane ? std::max<int64_t>(2048, (total + 455) / 456)
                      : (tc ? std::max<int64_t>(512, (total + 1215) / 1216) : std::max<int64_t>(256, (total + 2047) / 2048));
    B = (B + 63) / 64 * 64;
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
    plan.pairs_tested = total * (int64_t)T[0] * T[1] * T[2];
    // device copies: axes, item starts, items
    const size_t axb = sizeof(double) * (size_t)(L.n[0] + L.n[1] + L.n[2]);
    const size_t sb = sizeof(int32_t) * item_start.size(), ib = sizeof(int4) * std::max<size_t>(items.size(), 1);
    FGA_TRY(ws.tiles.ensure(axb + sb));
    FGA_TRY(ws.items.ensure(ib));
    FGA_TRY(ws.h_tiles.ensure(axb + sb));
    FGA_TRY(ws.h_items.ensure(ib));
    char *h = ws.h_tiles.as<char>();
    size_t off = 0;
    for (int d = 0; d < 3; d++) {
        std::memcpy(h + off, L.axis[d], sizeof(double) * (size_t)L.n[d]);
        off += sizeof(double) * (size_t)L.n[d];
    }
    std::memcpy(h + axb, item_start.data(), sb);
    if (!items.empty()) std::memcpy(ws.h_items.p, items.data(), sizeof(int4) * items.size());
    FGA_CUDA(cudaMemcpyAsync(ws.tiles.p, ws.h_tiles.p, axb + sb, cudaMemcpyHostToDevice, s));
    if (!items.empty()) FGA_CUDA(cudaMemcpyAsync(ws.items.p, ws.h_items.p, sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s));
    const double *dax = ws.tiles.as<double>();
    plan.ax[0] = dax;
    plan.ax[1] = dax + L.n[0];
    plan.ax[2] = dax + L.n[0] + L.n[1];
    plan.item_start = reinterpret_cast<const int32_t *>(ws.tiles.as<char>() + axb);
    plan.items = ws.items.as<int4>();
    return FGA_OK;
}

template <typename R>
static fga_status run_lattice_t(Workspace &ws, const LatticePlan &plan, const void *rec, double k, double rw, void *u,
                                cudaStream_t s, int cat) {
    const int TP = plan.T[0] * plan.T[1] * plan.T[2];
    // batch capacity: up to 64 beams, within ~72 KB of shared memory
    LatSmem L;
    int nb = 64;
    for (; nb > 8; nb -= 8) {
        L.init<R>(nb, plan.T[0], plan.T[1], plan.T[2]);
        if (L.bytes <= 72 * 1024) break;
    }
    L.init<R>(nb, plan.T[0], plan.T[1], plan.T[2]);
    FGA_TRY(ws.partial.ensure(sizeof(R) * 6 * (size_t)TP * (size_t)std::max(plan.nitems, 1)));
    const int cnt = prof_counting() ? 1 : 0;
    prof_add_pairs_tested(plan.pairs_tested);
    if (plan.nitems > 0) {
        const int pts = (L.nblocks() + 7) / 8;  // warp blocks per warp
        if (pts > 4) {
            set_error("lattice tile has more than 32 warp blocks");
            return FGA_ERR_UNSUPPORTED;
        }
        ProfScope ps(cat, s);
#define FGA_LAT2(PTS, CNT)                                                                                          \
    do {                                                                                                            \
        FGA_CUDA(cudaFuncSetAttribute(lattice_gather_kernel<R, PTS, CNT>,                                           \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes));                 \
        lattice_gather_kernel<R, PTS, CNT><<<plan.nitems, 256, L.bytes, s>>>(                                      \
            (const R *)rec, plan.ax[0], plan.ax[1], plan.ax[2], plan.n[0], plan.n[1], plan.n[2], L, plan.nt[1],    \
            plan.nt[2], plan.items, (R)k, (R)(rw * rw), ws.partial.as<R>());                                        \
    } while (0)
#define FGA_LAT(PTS)            \
    do {                        \
        if (cnt)                \
            FGA_LAT2(PTS, true);  \
        else                    \
            FGA_LAT2(PTS, false); \
    } while (0)
        if (pts == 1) FGA_LAT(1);
        else if (pts == 2) FGA_LAT(2);
        else if (pts == 3) FGA_LAT(3);
        else FGA_LAT(4);
#undef FGA_LAT
#undef FGA_LAT2
        FGA_CUDA(cudaGetLastError());
    }
    const int64_t total = (int64_t)plan.n[0] * plan.n[1] * plan.n[2];
    ProfScope ps(P_REDUCE, s);
    lattice_reduce_kernel<R><<<(unsigned)((total * 32 + 255) / 256), 256, 0, s>>>(
        ws.partial.as<R>(), plan.item_start, plan.n[0], plan.n[1], plan.n[2], plan.T[0], plan.T[1], plan.T[2],
        plan.nt[1], plan.nt[2], (R *)u);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

fga_status lattice_reduce_f32(const float *partial, const LatticePlan &plan, void *u, cudaStream_t s) {
    const int64_t total = (int64_t)plan.n[0] * plan.n[1] * plan.n[2];
    ProfScope ps(P_REDUCE, s);
    lattice_reduce_kernel<float><<<(unsigned)((total * 32 + 255) / 256), 256, 0, s>>>(
        partial, plan.item_start, plan.n[0], plan.n[1], plan.n[2], plan.T[0], plan.T[1], plan.T[2], plan.nt[1],
        plan.nt[2], (float *)u);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

// FP32: the tensor-core kernel (plans built with tc = true); FP64: the CUDA-core kernel
fga_status run_lattice(Workspace &ws, const LatticePlan &plan, int precision, const void *rec, double k, double rw,
                       void *u, cudaStream_t s, int cat, const float *amax) {
    if (precision == FGA_PREC_FP64) return run_lattice_t<double>(ws, plan, rec, k, rw, u, s, cat);
    if (plane_tc_eligible(plan)) return run_plane_tc(ws, plan, rec, k, rw, u, s, cat, amax);
    return run_lattice_tc(ws, plan, rec, k, rw, u, s, cat, amax);
}

}  // namespace fga
