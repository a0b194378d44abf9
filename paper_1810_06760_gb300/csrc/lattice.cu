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

template <typename R, int T0, int T1, int T2, int NBB>
__global__ void __launch_bounds__(256) lattice_gather_kernel(const R *__restrict__ rec, const double *__restrict__ ax0,
                                                            const double *__restrict__ ax1, const double *__restrict__ ax2,
                                                            int n0, int n1, int n2, int nt1, int nt2,
                                                            const int4 *__restrict__ items, R k, R rw2,
                                                            R *__restrict__ partial, int count_pairs) {
    constexpr int T12 = T1 * T2, TP = T0 * T12, PTS = (TP + 255) / 256;
    __shared__ R s_ae0[NBB][T0][6];  // A_c * E0(x_i)
    __shared__ R s_d0[NBB][T0];      // (x_i - Q_0)^2
    __shared__ R s_e12[NBB][T12][2]; // E1(x_j) E2(x_l)
    __shared__ R s_d12[NBB][T12];    // (x_j - Q_1)^2 + (x_l - Q_2)^2
    __shared__ R s_e1[NBB][T1][2], s_e2[NBB][T2][2], s_d1[NBB][T1], s_d2[NBB][T2];
    __shared__ R s_rec[NBB][REC];
    __shared__ R s_x[T0 + T1 + T2];
    __shared__ int s_nb;
    __shared__ unsigned s_pairs;

    const int4 it = items[blockIdx.x];
    const int t = it.x;
    const int tt0 = t / (nt1 * nt2), tt1 = (t / nt2) % nt1, tt2 = t % nt2;
    const int i0 = tt0 * T0, j0 = tt1 * T1, l0 = tt2 * T2;
    const int e0 = min(T0, n0 - i0), e1 = min(T1, n1 - j0), e2 = min(T2, n2 - l0);
    const int tid = threadIdx.x;
    // tile coordinates (ragged tiles repeat their last coordinate; those points are not written)
    if (tid < T0) s_x[tid] = (R)ax0[i0 + min(tid, e0 - 1)];
    else if (tid < T0 + T1) s_x[tid] = (R)ax1[j0 + min(tid - T0, e1 - 1)];
    else if (tid < T0 + T1 + T2) s_x[tid] = (R)ax2[l0 + min(tid - T0 - T1, e2 - 1)];
    if (tid == 0) s_pairs = 0;
    __syncthreads();
    const R lo0 = s_x[0], hi0 = s_x[T0 - 1], lo1 = s_x[T0], hi1 = s_x[T0 + T1 - 1];
    const R lo2 = s_x[T0 + T1], hi2 = s_x[T0 + T1 + T2 - 1];

    R acc[PTS][6];
#pragma unroll
    for (int q = 0; q < PTS; q++)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[q][c] = R(0);
    unsigned mine = 0;
    const R hk = R(-0.5) * k;

    for (int64_t base = it.y; base < it.z; base += NBB) {
        // 1. load up to NBB candidate records; keep those within rw of the tile's box
        if (tid < 32) {
            const int64_t b = base + tid;
            bool keep = false;
            R r[REC];
            if (tid < NBB && b < it.z) {
#pragma unroll
                for (int q = 0; q < REC; q++) r[q] = rec[b * REC + q];
                const R g0 = fmax(fmax(lo0 - r[0], r[0] - hi0), R(0));
                const R g1 = fmax(fmax(lo1 - r[1], r[1] - hi1), R(0));
                const R g2 = fmax(fmax(lo2 - r[2], r[2] - hi2), R(0));
                keep = g0 * g0 + g1 * g1 + g2 * g2 <= rw2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int slot = __popc(m & ((1u << tid) - 1u));
#pragma unroll
                for (int q = 0; q < REC; q++) s_rec[slot][q] = r[q];
            }
            if (tid == 0) s_nb = __popc(m);
        }
        __syncthreads();
        const int nb = s_nb;
        if (nb == 0) {
            __syncthreads();
            continue;
        }
        // 2. per-axis factors of the kept beams
        for (int e = tid; e < nb * (T0 + T1 + T2); e += 256) {
            const int b = e / (T0 + T1 + T2), a = e % (T0 + T1 + T2);
            const int d = a < T0 ? 0 : (a < T0 + T1 ? 1 : 2);
            const R dx = s_x[a] - s_rec[b][d];
            R er, ei;
            gauss_phase_exp<R>(k * s_rec[b][3 + d] * dx, hk * dx * dx, &er, &ei);
            if (d == 0) {
                s_d0[b][a] = dx * dx;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const R ar = s_rec[b][6 + 2 * c], ai = s_rec[b][7 + 2 * c];
                    s_ae0[b][a][2 * c] = ar * er - ai * ei;
                    s_ae0[b][a][2 * c + 1] = ar * ei + ai * er;
                }
            } else if (d == 1) {
                s_d1[b][a - T0] = dx * dx;
                s_e1[b][a - T0][0] = er;
                s_e1[b][a - T0][1] = ei;
            } else {
                s_d2[b][a - T0 - T1] = dx * dx;
                s_e2[b][a - T0 - T1][0] = er;
                s_e2[b][a - T0 - T1][1] = ei;
            }
        }
        __syncthreads();
        for (int e = tid; e < nb * T12; e += 256) {
            const int b = e / T12, jl = e % T12, j = jl / T2, l = jl % T2;
            const R ar = s_e1[b][j][0], ai = s_e1[b][j][1], br = s_e2[b][l][0], bi = s_e2[b][l][1];
            s_e12[b][jl][0] = ar * br - ai * bi;
            s_e12[b][jl][1] = ar * bi + ai * br;
            s_d12[b][jl] = s_d1[b][j] + s_d2[b][l];
        }
        __syncthreads();
        // 3. every thread adds the kept beams to its points
#pragma unroll
        for (int q = 0; q < PTS; q++) {
            const int p = tid + 256 * q;
            if (p < TP) {
                const int i = p / T12, jl = p % T12;
                const unsigned valid = (i < e0 && jl / T2 < e1 && jl % T2 < e2) ? 1u : 0u;
                for (int b = 0; b < nb; b++) {
                    const R d2 = s_d0[b][i] + s_d12[b][jl];
                    if (d2 <= rw2) {
                        mine += valid;
                        const R er = s_e12[b][jl][0], ei = s_e12[b][jl][1];
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const R ar = s_ae0[b][i][2 * c], ai = s_ae0[b][i][2 * c + 1];
                            acc[q][2 * c] += ar * er - ai * ei;
                            acc[q][2 * c + 1] += ar * ei + ai * er;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PTS; q++) {
        const int p = tid + 256 * q;
        if (p < TP) {
            R *dst = partial + ((int64_t)blockIdx.x * TP + p) * 6;
#pragma unroll
            for (int c = 0; c < 6; c++) dst[c] = acc[q][c];
        }
    }
    if (count_pairs) {
        atomicAdd(&s_pairs, mine);
        __syncthreads();
        if (tid == 0) atomicAdd(&g_lattice_pairs, (unsigned long long)s_pairs);
    }
}

template <typename R, int T0, int T1, int T2>
__global__ void lattice_reduce_kernel(const R *__restrict__ partial, const int32_t *__restrict__ item_start, int n0,
                                      int n1, int n2, int nt1, int nt2, R *__restrict__ u) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n0 * n1 * n2;
    if (g >= total) return;
    const int l = (int)(g % n2), j = (int)((g / n2) % n1), i = (int)(g / ((int64_t)n1 * n2));
    const int t = ((i / T0) * nt1 + j / T1) * nt2 + l / T2;
    const int p = ((i % T0) * T1 + j % T1) * T2 + l % T2;
    constexpr int TP = T0 * T1 * T2;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int it = item_start[t]; it < item_start[t + 1]; it++)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += (double)partial[((int64_t)it * TP + p) * 6 + c];
#pragma unroll
    for (int c = 0; c < 6; c++) u[g * 6 + c] = (R)acc[c];
}

// tile shapes: planes (one point along axis 2) use 16 x 16 x 1, volumes 8 x 8 x 8
static void tile_shape(const fga_lattice &L, int T[3]) {
    if (L.n[2] == 1) {
        T[0] = 16;
        T[1] = 16;
        T[2] = 1;
    } else {
        T[0] = T[1] = T[2] = 8;
    }
}

fga_status build_lattice_plan(Workspace &ws, const BinGrid &g, const int32_t *cell_start_dev, const fga_lattice &L,
                              cudaStream_t s, LatticePlan &plan) {
    int T[3];
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
    int64_t B = std::max<int64_t>(256, (total + 4095) / 4096);
    B = (B + 31) / 32 * 32;
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

template <typename R, int T0, int T1, int T2>
static fga_status run_lattice_t(Workspace &ws, const LatticePlan &plan, const void *rec, double k, double rw, void *u,
                                cudaStream_t s) {
    constexpr int TP = T0 * T1 * T2;
    constexpr int NBB = sizeof(R) == 4 ? 32 : 16;
    FGA_TRY(ws.partial.ensure(sizeof(R) * 6 * (size_t)TP * (size_t)std::max(plan.nitems, 1)));
    const int cnt = prof_counting() ? 1 : 0;
    prof_add_pairs_tested(plan.pairs_tested);
    if (plan.nitems > 0) {
        ProfScope ps(P_GATHER, s);
        lattice_gather_kernel<R, T0, T1, T2, NBB><<<plan.nitems, 256, 0, s>>>(
            (const R *)rec, plan.ax[0], plan.ax[1], plan.ax[2], plan.n[0], plan.n[1], plan.n[2], plan.nt[1], plan.nt[2],
            plan.items, (R)k, (R)(rw * rw), ws.partial.as<R>(), cnt);
        FGA_CUDA(cudaGetLastError());
    }
    const int64_t total = (int64_t)plan.n[0] * plan.n[1] * plan.n[2];
    ProfScope ps(P_REDUCE, s);
    lattice_reduce_kernel<R, T0, T1, T2><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
        ws.partial.as<R>(), plan.item_start, plan.n[0], plan.n[1], plan.n[2], plan.nt[1], plan.nt[2], (R *)u);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

fga_status run_lattice(Workspace &ws, const LatticePlan &plan, int precision, const void *rec, double k, double rw,
                       void *u, cudaStream_t s) {
    const bool plane = plan.T[2] == 1;
    if (precision == FGA_PREC_FP64)
        return plane ? run_lattice_t<double, 16, 16, 1>(ws, plan, rec, k, rw, u, s)
                     : run_lattice_t<double, 8, 8, 8>(ws, plan, rec, k, rw, u, s);
    return plane ? run_lattice_t<float, 16, 16, 1>(ws, plan, rec, k, rw, u, s)
                 : run_lattice_t<float, 8, 8, 8>(ws, plan, rec, k, rw, u, s);
}

}  // namespace fga
