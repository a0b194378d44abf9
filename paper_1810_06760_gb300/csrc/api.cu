// C ABI of the library (include/fga.h): handles, argument checks, and the solve orchestration.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "fga_beam.cuh"
#include "gather.cuh"

namespace fga {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

fga_status cuda_fail(cudaError_t e, const char *what) {
    char buf[512];
    std::snprintf(buf, sizeof buf, "CUDA error %d (%s: %s) in %s", (int)e, cudaGetErrorName(e), cudaGetErrorString(e),
                  what);
    g_err = buf;
    return e == cudaErrorMemoryAllocation ? FGA_ERR_OOM : FGA_ERR_CUDA;
}

// Per-thread block cache.  Off by default: every DevBuf/HostBuf then maps to cudaMalloc/cudaFree
// (whose implicit device synchronisation also orders reuse).  A thread that issues all its work on
// one stream (a server worker) turns it on: released blocks go to the thread's cache and are handed
// back to later allocations of the same thread, whose work is ordered after every earlier use on
// that stream, so no allocation or free stalls the other streams.  Pinned host blocks are cached only
// after the stream has drained (the host writes into them).
namespace {
struct BlockCache {
    bool on = false;
    cudaStream_t stream = nullptr;
    std::multimap<size_t, void *> dev, host;
    size_t dev_bytes = 0, host_bytes = 0;
};
thread_local BlockCache tl_cache;
// a cached block of at least need bytes and not much larger; its size goes to *size
void *cache_take(std::multimap<size_t, void *> &c, size_t &total, size_t need, size_t *size) {
    auto it = c.lower_bound(need);
    if (it == c.end() || it->first > 2 * need + ((size_t)1 << 20)) return nullptr;
    void *p = it->second;
    *size = it->first;
    total -= it->first;
    c.erase(it);
    return p;
}
}  // namespace

// device bytes held by the library's own buffers, and the caller's bound on them (0: none)
std::atomic<int64_t> g_dev_bytes{0}, g_dev_limit{0};

static cudaError_t dev_alloc(void **p, size_t need) {
    const int64_t lim = g_dev_limit.load();
    if (lim > 0 && g_dev_bytes.load() + (int64_t)need > lim) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, need);
    if (e == cudaSuccess) g_dev_bytes += (int64_t)need;
    return e;
}
static void dev_free(void *p, size_t bytes) {
    cudaFree(p);
    g_dev_bytes -= (int64_t)bytes;
}

void block_cache_enable(cudaStream_t s) {
    tl_cache.on = true;
    tl_cache.stream = s;
}
size_t block_cache_bytes() { return tl_cache.dev_bytes; }
void block_cache_trim(size_t keep) {
    // largest blocks first
    while (tl_cache.dev_bytes > keep && !tl_cache.dev.empty()) {
        auto it = std::prev(tl_cache.dev.end());
        dev_free(it->second, it->first);
        tl_cache.dev_bytes -= it->first;
        tl_cache.dev.erase(it);
    }
}
void block_cache_disable() {
    block_cache_trim(0);
    for (auto &kv : tl_cache.host) cudaFreeHost(kv.second);
    tl_cache.host.clear();
    tl_cache.host_bytes = 0;
    tl_cache.on = false;
    tl_cache.stream = nullptr;
}

fga_status DevBuf::ensure(size_t need) {
    if (need <= bytes && p) return FGA_OK;
    release();
    if (need == 0) need = 16;
    if (tl_cache.on) {
        size_t got = 0;
        if (void *q = cache_take(tl_cache.dev, tl_cache.dev_bytes, need, &got)) {
            p = q;
            bytes = got;
            return FGA_OK;
        }
    }
    cudaError_t e = dev_alloc(&p, need);
    if (e == cudaErrorMemoryAllocation && tl_cache.on && tl_cache.dev_bytes > 0) {
        cudaGetLastError();
        block_cache_trim(0);
        e = dev_alloc(&p, need);
    }
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        cudaGetLastError();
        char buf[160];
        std::snprintf(buf, sizeof buf, "device allocation of %zu bytes failed (%s)", need, cudaGetErrorString(e));
        set_error(buf);
        return FGA_ERR_OOM;
    }
    bytes = need;
    return FGA_OK;
}
void DevBuf::release() {
    if (p) {
        if (tl_cache.on) {
            tl_cache.dev.emplace(bytes, p);
            tl_cache.dev_bytes += bytes;
        } else {
            dev_free(p, bytes);
        }
    }
    p = nullptr;
    bytes = 0;
}
fga_status HostBuf::ensure(size_t need) {
    if (need <= bytes && p) return FGA_OK;
    release();
    if (need == 0) need = 16;
    if (tl_cache.on) {
        size_t got = 0;
        if (void *q = cache_take(tl_cache.host, tl_cache.host_bytes, need, &got)) {
            p = q;
            bytes = got;
            return FGA_OK;
        }
    }
    cudaError_t e = cudaMallocHost(&p, need);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        cudaGetLastError();
        set_error("pinned host allocation failed");
        return FGA_ERR_OOM;
    }
    bytes = need;
    return FGA_OK;
}
void HostBuf::release() {
    if (p) {
        if (tl_cache.on) {
            cudaStreamSynchronize(tl_cache.stream);
            tl_cache.host.emplace(bytes, p);
            tl_cache.host_bytes += bytes;
        } else {
            cudaFreeHost(p);
        }
    }
    p = nullptr;
    bytes = 0;
}
void Workspace::release() {
    for (DevBuf *d : {&keys, &keys_alt, &vals, &vals_alt, &hist, &scan_blocks, &cell_start, &rec, &items, &tiles,
                      &partial, &pts, &status, &rec_amax})
        d->release();
    for (HostBuf *h : {&h_cell_start, &h_items, &h_tiles}) h->release();
}

// pack the 10 node fields into 3 float4 per node
__global__ void pack_grid_kernel(const float *__restrict__ src, float4 *__restrict__ dst, int64_t nn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const float *s = src + i * 10;
    dst[3 * i] = make_float4(s[0], s[1], s[2], s[3]);
    dst[3 * i + 1] = make_float4(s[4], s[5], s[6], s[7]);
    dst[3 * i + 2] = make_float4(s[8], s[9], 0.f, 0.f);
}

__global__ void max_field0_kernel(const float4 *__restrict__ g, int64_t nn, unsigned *__restrict__ out) {
    __shared__ unsigned sm;
    if (threadIdx.x == 0) sm = 0;
    __syncthreads();
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(g[3 * i].x));
    atomicMax(&sm, __float_as_uint(m));  // non-negative floats order like their bit patterns
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(out, sm);
}

static double sample_hermite_margin(double cmax, double dt, int w) { return cmax * std::fabs(dt) * (w + 1.0); }

// profiling state (process-wide; the profiling calls are meant for one host thread)
struct ProfState {
    int mode = 0;  // 0 off, 1 counters, 2 counters + event times
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_cat;
    size_t used = 0;
    int64_t launches = 0, count[P_NCAT] = {};
    double ms[P_NCAT] = {};
    int64_t beam_steps = 0, pairs_tested = 0;
    void fold() {  // accumulate the recorded event pairs
        for (size_t i = 0; i + 1 < used; i += 2) {
            float t = 0.f;
            if (cudaEventSynchronize(ev[i + 1]) == cudaSuccess && cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess)
                ms[ev_cat[i]] += t;
            else
                cudaGetLastError();
        }
        used = 0;
    }
};
static ProfState g_prof;

ProfScope::ProfScope(int cat, cudaStream_t st) : idx(-1), s(st) {
    if (g_prof.mode == 0) return;
    g_prof.launches++;
    g_prof.count[cat]++;
    if (g_prof.mode < 2) return;
    if (g_prof.used + 2 > 8192) g_prof.fold();
    while (g_prof.ev.size() < g_prof.used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        g_prof.ev.push_back(e);
        g_prof.ev_cat.push_back(0);
    }
    idx = (int)g_prof.used;
    g_prof.used += 2;
    g_prof.ev_cat[idx] = cat;
    cudaEventRecord(g_prof.ev[idx], s);
}
ProfScope::~ProfScope() {
    if (idx >= 0) cudaEventRecord(g_prof.ev[idx + 1], s);
}
bool prof_counting() { return g_prof.mode == 1 || g_prof.mode == 3; }
void prof_add_beam_steps(int64_t n) {
    if (g_prof.mode) g_prof.beam_steps += n;
}
void prof_add_pairs_tested(int64_t n) {
    if (g_prof.mode) g_prof.pairs_tested += n;
}

}  // namespace fga

namespace fga {
// x = (r cos(theta) cos(phi), r sin(theta) cos(phi), r sin(phi)) for points (r, theta, phi) (Sec. 3)
__global__ void spherical_to_cartesian_kernel(const double *__restrict__ rtp, int64_t n, double *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = rtp[3 * i], th = rtp[3 * i + 1], ph = rtp[3 * i + 2];
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    x[3 * i] = r * ct * cp;
    x[3 * i + 1] = r * st * cp;
    x[3 * i + 2] = r * sp;
}

fga_status spherical_points(const double *rtp, int64_t n, DevBuf &out, cudaStream_t s) {
    FGA_TRY(out.ensure(sizeof(double) * 3 * (size_t)std::max<int64_t>(n, 1)));
    if (n > 0) {
        spherical_to_cartesian_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rtp, n, out.as<double>());
        FGA_CUDA(cudaGetLastError());
    }
    return FGA_OK;
}

fga_status cartesian_desc(const fga_solve_desc *sd, fga_solve_desc &out, DevBuf &rx, DevBuf &snap, cudaStream_t s) {
    out = *sd;
    if (sd->coords == FGA_COORDS_CARTESIAN) return FGA_OK;
    FGA_CHECK(sd->coords == FGA_COORDS_SPHERICAL, "solve descriptor: coords must be FGA_COORDS_CARTESIAN or _SPHERICAL");
    FGA_CHECK(!sd->rx_lattice && !sd->snap_lattice, "solve descriptor: lattices take Cartesian coordinates only");
    if (sd->n_rx > 0 && sd->rx) {
        FGA_TRY(spherical_points(sd->rx, sd->n_rx, rx, s));
        out.rx = rx.as<double>();
    }
    if (sd->n_snap > 0 && sd->snap) {
        FGA_TRY(spherical_points(sd->snap, sd->n_snap, snap, s));
        out.snap = snap.as<double>();
    }
    out.coords = FGA_COORDS_CARTESIAN;
    return FGA_OK;
}

fga_status sync_layered_count(fga_beams *b, cudaStream_t s) {
    if (!b->layered) return FGA_OK;
    unsigned long long c[2] = {0, 0};
    FGA_CUDA(cudaMemcpyAsync(c, b->counts.p, sizeof c, cudaMemcpyDeviceToHost, s));
    FGA_CUDA(cudaStreamSynchronize(s));
    b->nb = (int64_t)std::min<unsigned long long>(c[0], (unsigned long long)b->cap);
    return FGA_OK;
}
}  // namespace fga

using namespace fga;

extern "C" {

void fga_last_error(char *buf, size_t cap) {
    if (!buf || cap == 0) return;
    std::snprintf(buf, cap, "%s", g_err.c_str());
}

int fga_version(void) { return 10000; }

fga_status fga_set_device_memory_limit(double bytes) {
    g_dev_limit.store(bytes > 0 ? (int64_t)bytes : 0);
    return FGA_OK;
}

double fga_device_memory_in_use(void) { return (double)g_dev_bytes.load(); }

fga_status fga_model_create(fga_model **out, const fga_model_desc *d, const float *grid_p, const float *grid_s,
                            fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(out && d, "fga_model_create: NULL argument");
    FGA_CHECK(d->kind >= FGA_MEDIUM_CONST && d->kind <= FGA_MEDIUM_LAYERED, "fga_model_create: bad medium kind");
    fga_model *m = new fga_model();
    std::memset(&m->dev, 0, sizeof(m->dev));
    m->dev.kind = d->kind;
    m->dev.cp0 = d->cp0;
    m->dev.cs0 = d->cs0;
    m->dev.amp = d->amp;
    m->dev.cs_ratio = d->cs_ratio;
    if (d->kind == FGA_MEDIUM_CONST) {
        if (!(d->cp0 > 0 && d->cs0 > 0)) {
            delete m;
            set_error("fga_model_create: constant speeds must be > 0");
            return FGA_ERR_INVALID_ARG;
        }
        m->cmax[0] = d->cp0;
        m->cmax[1] = d->cs0;
    } else if (d->kind == FGA_MEDIUM_SINE) {
        if (!(d->cp0 > std::fabs(d->amp) && d->cs_ratio > 0)) {
            delete m;
            set_error("fga_model_create: sine medium needs cp0 > |amp| and cs_ratio > 0");
            return FGA_ERR_INVALID_ARG;
        }
        m->cmax[0] = d->cp0 + std::fabs(d->amp);
        m->cmax[1] = m->cmax[0] * d->cs_ratio;
    } else if (d->kind == FGA_MEDIUM_GRID) {
        bool ok = grid_p && grid_s;
        for (int a = 0; a < 3; a++) ok = ok && d->n[a] >= 2 && d->spacing[a] > 0;
        if (!ok) {
            delete m;
            set_error("fga_model_create: grid needs n >= 2 per axis, spacing > 0 and both field arrays");
            return FGA_ERR_INVALID_ARG;
        }
        const int64_t nn = (int64_t)d->n[0] * d->n[1] * d->n[2];
        fga_status st = m->grid.ensure(sizeof(float4) * 3 * 2 * (size_t)nn);
        if (st != FGA_OK) {
            delete m;
            return st;
        }
        float4 *gp = m->grid.as<float4>(), *gs = gp + 3 * nn;
        const unsigned blocks = (unsigned)((nn + 255) / 256);
        pack_grid_kernel<<<blocks, 256, 0, s>>>(grid_p, gp, nn);
        pack_grid_kernel<<<blocks, 256, 0, s>>>(grid_s, gs, nn);
        unsigned *dmax = nullptr;
        cudaError_t e = cudaMalloc(&dmax, 2 * sizeof(unsigned));
        unsigned hmax[2] = {0, 0};
        if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned), s);
        if (e == cudaSuccess) {
            max_field0_kernel<<<304, 256, 0, s>>>(gp, nn, dmax);
            max_field0_kernel<<<304, 256, 0, s>>>(gs, nn, dmax + 1);
            e = cudaMemcpyAsync(hmax, dmax, sizeof hmax, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (dmax) cudaFree(dmax);
        if (e != cudaSuccess) {
            delete m;
            return cuda_fail(e, "fga_model_create");
        }
        float fm[2];
        std::memcpy(fm, hmax, sizeof fm);
        m->cmax[0] = fm[0];
        m->cmax[1] = fm[1];
        m->dev.gp = gp;
        m->dev.gs = gs;
        for (int a = 0; a < 3; a++) {
            m->dev.n[a] = d->n[a];
            m->dev.o[a] = d->origin[a];
            m->dev.h[a] = d->spacing[a];
            m->dev.inv_h[a] = 1.0 / d->spacing[a];
        }
    } else {
        bool ok = d->nlayers >= 1 && d->nlayers <= MAX_LAYERS && d->layer_cp && d->layer_cs && d->layer_rho &&
                  (d->nlayers == 1 || d->z_interfaces);
        if (!ok) {
            delete m;
            set_error("fga_model_create: layered medium needs 1..8 layers and their arrays");
            return FGA_ERR_INVALID_ARG;
        }
        const bool spheres = d->layer_shape == FGA_LAYERS_SPHERES, undul = d->layer_shape == FGA_LAYERS_UNDULATING;
        const double *nv = d->layer_normal;
        const double nn = std::sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
        const char *bad = nullptr;
        if (d->layer_shape != FGA_LAYERS_PLANES && !spheres && !undul)
            bad = "fga_model_create: layer_shape must be FGA_LAYERS_PLANES, _SPHERES or _UNDULATING";
        else if (!std::isfinite(nn))
            bad = "fga_model_create: layer_normal is not finite";
        else if ((spheres || undul) && nn != 0.0)
            bad = "fga_model_create: curved layers take no layer_normal";
        else if (undul && !(d->layer_wavelength[0] > 0.0 && d->layer_wavelength[1] > 0.0 &&
                            std::isfinite(d->layer_wavelength[0]) && std::isfinite(d->layer_wavelength[1])))
            bad = "fga_model_create: undulating layers need finite wavelengths > 0";
        else if (spheres && !(std::isfinite(d->layer_center[0]) && std::isfinite(d->layer_center[1]) &&
                              std::isfinite(d->layer_center[2])))
            bad = "fga_model_create: layer_center is not finite";
        for (int l = 0; !bad && l < d->nlayers; l++)
            if (!(std::isfinite(d->layer_cp[l]) && d->layer_cs[l] > 0.0 && d->layer_cp[l] > d->layer_cs[l] &&
                  d->layer_rho[l] > 0.0 && std::isfinite(d->layer_rho[l])))
                bad = "fga_model_create: every layer needs finite c_p > c_s > 0 and rho > 0";
        for (int l = 0; !bad && l + 1 < d->nlayers; l++) {
            const double z = d->z_interfaces[l];
            if (!std::isfinite(z) || (spheres && !(z > 0.0)))
                bad = "fga_model_create: interface depths must be finite (radii positive)";
            else if (l > 0 && (spheres ? !(z < d->z_interfaces[l - 1]) : !(z > d->z_interfaces[l - 1])))
                bad = spheres ? "fga_model_create: sphere radii must decrease strictly"
                              : "fga_model_create: interface depths must increase strictly";
            else if (undul && !std::isfinite(d->layer_amp[l]))
                bad = "fga_model_create: layer_amp is not finite";
            else if (undul && l > 0 &&
                     !(std::fabs(d->layer_amp[l - 1]) + std::fabs(d->layer_amp[l]) < z - d->z_interfaces[l - 1]))
                bad = "fga_model_create: neighbouring undulating interfaces may touch";
        }
        if (bad) {
            delete m;
            set_error(bad);
            return FGA_ERR_INVALID_ARG;
        }
        m->dev.nlay = d->nlayers;
        m->cmax[0] = m->cmax[1] = 0;
        for (int l = 0; l < d->nlayers; l++) {
            m->dev.lcp[l] = d->layer_cp[l];
            m->dev.lcs[l] = d->layer_cs[l];
            m->dev.lrho[l] = d->layer_rho[l];
            m->cmax[0] = std::max(m->cmax[0], d->layer_cp[l]);
            m->cmax[1] = std::max(m->cmax[1], d->layer_cs[l]);
            // spheres: minus the radius, so that the depth -|x - centre| increases across the interfaces
            if (l + 1 < d->nlayers) m->dev.zif[l] = spheres ? -d->z_interfaces[l] : d->z_interfaces[l];
        }
        m->dev.shells = spheres ? 1 : 0;
        for (int c = 0; c < 3; c++) m->dev.ctr[c] = spheres ? d->layer_center[c] : 0.0;
        m->dev.undul = undul ? 1 : 0;
        for (int l = 0; l + 1 < d->nlayers; l++) m->dev.uamp[l] = undul ? d->layer_amp[l] : 0.0;
        for (int c = 0; c < 2; c++) m->dev.uk[c] = undul ? 2.0 * M_PI / d->layer_wavelength[c] : 0.0;
        // the layer frame of planar layers: third axis the normal (frame_from_normal)
        const double n3[3] = {nn > 0 ? nv[0] / nn : 0.0, nn > 0 ? nv[1] / nn : 0.0, nn > 0 ? nv[2] / nn : 1.0};
        m->dev.tilted = (n3[0] != 0.0 || n3[1] != 0.0 || n3[2] != 1.0) ? 1 : 0;
        if (m->dev.tilted) {
            frame_from_normal(n3, m->dev.R);
        } else {
            for (int c = 0; c < 9; c++) m->dev.R[c] = (c % 4 == 0) ? 1.0 : 0.0;
        }
    }
    m->dev.fill_f32();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        m->grid.release();
        delete m;
        return cuda_fail(e, "fga_model_create");
    }
    *out = m;
    return FGA_OK;
}

fga_status fga_model_destroy(fga_model *m) {
    if (!m) return FGA_OK;
    m->grid.release();
    delete m;
    return FGA_OK;
}

fga_status fga_decompose(const fga_model *m, const fga_init_desc *init, fga_beams **out, fga_stream_t s) {
    return decompose_impl(m, init, out, (cudaStream_t)s);
}

fga_status fga_transform(const fga_init_desc *init, void *F_out, fga_stream_t s) {
    return transform_impl(init, F_out, (cudaStream_t)s);
}

fga_status fga_propagate(const fga_model *m, fga_beams *b, double dt, int nsteps, fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(m && b, "fga_propagate: NULL argument");
    FGA_CHECK(nsteps >= 0 && std::isfinite(dt), "fga_propagate: nsteps >= 0 and a finite dt required");
    FGA_CHECK(b->layered == (m->dev.kind == FGA_MEDIUM_LAYERED), "fga_propagate: beams made for another kind of medium");
    if (b->layered) {
        FGA_TRY(launch_layered_steps(m, b, dt, nsteps, s));
        FGA_TRY(sync_layered_count(b, s));
    } else {
        for (int n0 = 0; n0 < nsteps; n0 += 64)
            FGA_TRY(launch_propagate(m, b, dt, std::min(64, nsteps - n0), nullptr, s));
    }
    b->last_stream = s;
    return FGA_OK;
}

// sort the beams' current centres on a grid; returns the permutation and the bucket starts (device)
static fga_status bin_beams(const fga_beams *b, const BinGrid &g, int32_t **perm, cudaStream_t s) {
    Workspace &ws = b->ws;
    const int nbk = 4 * (g.ncells + 1);
    FGA_TRY(ws.keys.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(b->nb, 1)));
    FGA_TRY(ws.cell_start.ensure(sizeof(int32_t) * (size_t)(nbk + 1)));
    const int kind = b->precision == FGA_PREC_FP64 ? Q_F64_SOA : Q_F32_SOA;
    FGA_TRY(bin_centres(g, b->state.p, kind, b->cap, b->nb, b->flags.as<int32_t>(), ws.keys.as<int32_t>(), s));
    return sort_keys_to_perm(ws, ws.keys.as<int32_t>(), b->nb, nbk, perm, ws.cell_start.as<int32_t>(), s);
}

static fga_status host_points(const double *x_dev, int64_t n, std::vector<double> &out, cudaStream_t s) {
    out.resize((size_t)(3 * n));
    if (n == 0) return FGA_OK;
    FGA_CUDA(cudaMemcpyAsync(out.data(), x_dev, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
    FGA_CUDA(cudaStreamSynchronize(s));
    for (double v : out)
        if (!std::isfinite(v)) {
            set_error("points must be finite");
            return FGA_ERR_INVALID_ARG;
        }
    return FGA_OK;
}

// Gaussian sum of the current state at points (records gathered in cell order, state untouched)
}  // extern "C"

namespace fga {
struct Mat3 {
    double a[9];
};

// tilted layered media: the sums run in the layer frame; the field vectors come back as R^T u'
template <typename R>
__global__ void layer_frame_to_global_kernel(R *__restrict__ u, int64_t n, Mat3 Rm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R v[6];
    for (int f = 0; f < 6; f++) v[f] = u[6 * i + f];
    for (int c = 0; c < 3; c++) {
        R re = 0, im = 0;
        for (int j = 0; j < 3; j++) {
            re += (R)Rm.a[3 * j + c] * v[2 * j];
            im += (R)Rm.a[3 * j + c] * v[2 * j + 1];
        }
        u[6 * i + 2 * c] = re;
        u[6 * i + 2 * c + 1] = im;
    }
}
}  // namespace fga

extern "C" {

static fga_status reconstruct_now_frame(const fga_beams *b, const double *x_dev, const std::vector<double> &xh,
                                        int64_t n, double rw, void *u_out, cudaStream_t s);

static fga_status reconstruct_now(const fga_beams *b, const double *x_dev, const std::vector<double> &xh, int64_t n,
                                  double rw, void *u_out, cudaStream_t s) {
    if (n == 0) return FGA_OK;
    if (b->tilted) return reconstruct_now_frame(b, x_dev, xh, n, rw, u_out, s);
    Workspace &ws = b->ws;
    const BinGrid g = make_grid(xh.data(), n, rw);
    int32_t *perm = nullptr;
    FGA_TRY(bin_beams(b, g, &perm, s));
    SumPlan plan;
    FGA_TRY(build_sum_plan(ws, g, ws.cell_start.as<int32_t>(), 4, xh.data(), n, s, plan));  // syncs
    const size_t rb = b->precision == FGA_PREC_FP64 ? 8 : 4;
    FGA_TRY(ws.rec.ensure(rb * REC * (size_t)std::max<int64_t>(plan.n_rec, 1)));
    FGA_TRY(launch_records_from_state(b, perm, plan.beg, plan.n_in, plan.rec_off, ws.rec.p, s));
    return run_sum(ws, plan, b->precision, ws.rec.p, x_dev, b->k, rw, u_out, s, P_GATHER_STATE);
}

static fga_status check_lattice(const fga_lattice *L, const char *who) {
    for (int d = 0; d < 3; d++) {
        if (L->n[d] < 1 || !L->axis[d]) {
            set_error(std::string(who) + ": lattice axes need n >= 1 and a coordinate array");
            return FGA_ERR_INVALID_ARG;
        }
        for (int i = 0; i < L->n[d]; i++)
            if (!std::isfinite(L->axis[d][i]) || (i > 0 && !(L->axis[d][i] > L->axis[d][i - 1]))) {
                set_error(std::string(who) + ": lattice coordinates must be finite and increasing");
                return FGA_ERR_INVALID_ARG;
            }
    }
    if ((int64_t)L->n[0] * L->n[1] * L->n[2] >= ((int64_t)1 << 31)) {
        set_error(std::string(who) + ": lattice too large");
        return FGA_ERR_INVALID_ARG;
    }
    return FGA_OK;
}

static std::vector<double> lattice_corners(const fga_lattice *L) {
    std::vector<double> c;
    for (int a = 0; a < 2; a++)
        for (int b2 = 0; b2 < 2; b2++)
            for (int e = 0; e < 2; e++) {
                c.push_back(L->axis[0][a ? L->n[0] - 1 : 0]);
                c.push_back(L->axis[1][b2 ? L->n[1] - 1 : 0]);
                c.push_back(L->axis[2][e ? L->n[2] - 1 : 0]);
            }
    return c;
}

// points into the layer frame (x' = R x), the sum there, the field vectors back to global coordinates
static fga_status reconstruct_now_frame(const fga_beams *b, const double *, const std::vector<double> &xh, int64_t n,
                                        double rw, void *u_out, cudaStream_t s) {
    std::vector<double> xr((size_t)(3 * n));
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < 3; c++)
            xr[(size_t)(3 * i + c)] = b->R[3 * c] * xh[(size_t)(3 * i)] + b->R[3 * c + 1] * xh[(size_t)(3 * i + 1)] +
                                      b->R[3 * c + 2] * xh[(size_t)(3 * i + 2)];
    ScopedDevBuf xd;
    FGA_TRY(xd.ensure(sizeof(double) * xr.size()));
    FGA_CUDA(cudaMemcpyAsync(xd.p, xr.data(), sizeof(double) * xr.size(), cudaMemcpyHostToDevice, s));
    fga_beams *bf = const_cast<fga_beams *>(b);
    bf->tilted = false;   // the sum itself is the flat one, in the layer frame
    const fga_status st = reconstruct_now(b, xd.as<double>(), xr, n, rw, u_out, s);
    bf->tilted = true;
    FGA_TRY(st);
    Mat3 Rm;
    for (int i = 0; i < 9; i++) Rm.a[i] = b->R[i];
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (b->precision == FGA_PREC_FP64)
        layer_frame_to_global_kernel<double><<<blocks, 256, 0, s>>>(static_cast<double *>(u_out), n, Rm);
    else
        layer_frame_to_global_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float *>(u_out), n, Rm);
    FGA_CUDA(cudaGetLastError());
    // the rotated points are released when this scope ends
    FGA_CUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

// lattice sum of the current state (records gathered in cell order, state untouched)
static fga_status reconstruct_lattice_now(const fga_beams *b, const fga_lattice *L, double rw, void *u_out,
                                          cudaStream_t s) {
    if (b->tilted) {
        // a lattice is not aligned with the layer frame: its points, x-major, as a point set
        const int64_t n = (int64_t)L->n[0] * L->n[1] * L->n[2];
        std::vector<double> xh((size_t)(3 * n));
        int64_t q = 0;
        for (int i = 0; i < L->n[0]; i++)
            for (int j = 0; j < L->n[1]; j++)
                for (int l = 0; l < L->n[2]; l++, q++) {
                    xh[(size_t)(3 * q)] = L->axis[0][i];
                    xh[(size_t)(3 * q + 1)] = L->axis[1][j];
                    xh[(size_t)(3 * q + 2)] = L->axis[2][l];
                }
        return reconstruct_now_frame(b, nullptr, xh, n, rw, u_out, s);
    }
    Workspace &ws = b->ws;
    const std::vector<double> corners = lattice_corners(L);
    const BinGrid g = make_grid(corners.data(), 8, rw);
    int32_t *perm = nullptr;
    FGA_TRY(bin_beams(b, g, &perm, s));
    LatticePlan plan;
    FGA_TRY(build_lattice_plan(ws, g, ws.cell_start.as<int32_t>(), *L, s, plan, b->precision == FGA_PREC_FP32, b->k,
                               rw));  // syncs
    const size_t rb = b->precision == FGA_PREC_FP64 ? 8 : 4;
    FGA_TRY(ws.rec.ensure(rb * REC * (size_t)std::max<int64_t>(plan.n_rec, 1)));
    FGA_TRY(launch_records_from_state(b, perm, plan.beg, plan.n_in, plan.rec_off, ws.rec.p, s));
    return run_lattice(ws, plan, b->precision, ws.rec.p, b->k, rw, u_out, s, P_GATHER_STATE);
}

fga_status fga_reconstruct_lattice(const fga_beams *b, const fga_lattice *lat, double rw, void *u_out,
                                   fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(b && lat && u_out, "fga_reconstruct_lattice: NULL argument");
    FGA_TRY(check_lattice(lat, "fga_reconstruct_lattice"));
    if (!(rw > 0)) rw = 6.0 / std::sqrt(b->k);
    FGA_TRY(sync_layered_count(const_cast<fga_beams *>(b), s));
    FGA_TRY(status_reset(b->ws, s));
    FGA_TRY(reconstruct_lattice_now(b, lat, rw, u_out, s));
    return status_check(b->ws, s, "fga_reconstruct_lattice");
}

fga_status fga_reconstruct(const fga_beams *b, const double *x, int64_t n, double rw, void *u_out, fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(b, "fga_reconstruct: NULL beams");
    FGA_CHECK(n >= 0, "fga_reconstruct: n < 0");
    if (n == 0) return FGA_OK;
    FGA_CHECK(x && u_out, "fga_reconstruct: NULL points or output");
    FGA_CHECK(n < ((int64_t)1 << 31), "fga_reconstruct: too many points");
    if (!(rw > 0)) rw = 6.0 / std::sqrt(b->k);
    std::vector<double> xh;
    FGA_TRY(host_points(x, n, xh, s));
    FGA_TRY(sync_layered_count(const_cast<fga_beams *>(b), s));
    return reconstruct_now(b, x, xh, n, rw, u_out, s);
}

fga_status fga_reconstruct_spherical(const fga_beams *b, const double *rtp, int64_t n, double rw, void *u_out,
                                     fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(b, "fga_reconstruct_spherical: NULL beams");
    FGA_CHECK(n >= 0, "fga_reconstruct_spherical: n < 0");
    if (n == 0) return FGA_OK;
    FGA_CHECK(rtp && u_out, "fga_reconstruct_spherical: NULL points or output");
    FGA_CHECK(n < ((int64_t)1 << 31), "fga_reconstruct_spherical: too many points");
    if (!(rw > 0)) rw = 6.0 / std::sqrt(b->k);
    ScopedDevBuf x;
    FGA_TRY(spherical_points(rtp, n, x, s));
    std::vector<double> xh;
    FGA_TRY(host_points(x.as<double>(), n, xh, s));   // synchronises s
    FGA_TRY(sync_layered_count(const_cast<fga_beams *>(b), s));
    FGA_TRY(reconstruct_now(b, x.as<double>(), xh, n, rw, u_out, s));
    FGA_CUDA(cudaStreamSynchronize(s));   // the converted points are released with this scope
    return FGA_OK;
}

fga_status fga_solve(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd, void *seis_out,
                     void *snap_out, fga_stream_t s_) {
    // records of up to 48 GB per window of steps (at most 40% of the free device memory): fewer windows,
    // so fewer sorts and fewer passes over the beam state
    return solve_impl(m, init, sd, seis_out, snap_out, (cudaStream_t)s_, 48.0e9, nullptr);
}

}  // extern "C"

namespace fga {
// a cancelled solve: its stream drained before the beam set is freed
static fga_status cancelled(cudaStream_t s) {
    cudaStreamSynchronize(s);
    set_error("the request was cancelled");
    return FGA_ERR_CANCELLED;
}

// non-finite values in the final beam state, the seismograms or the snapshot of a solve (status word 1)
static fga_status flag_solve_nonfinite(const fga_beams *b, const fga_solve_desc *sd, int64_t nrx, bool seis,
                                       const void *seis_out, const void *snap_out, cudaStream_t s) {
    Workspace &ws = b->ws;
    FGA_TRY(flag_nonfinite_state(ws, b->state.p, b->cap, b->nb, NF, b->precision, s));
    if (seis) FGA_TRY(flag_nonfinite(ws, seis_out, (int64_t)sd->n_times * nrx * 6, b->precision, s));
    const fga_lattice *snL = sd->snap_lattice;
    const int64_t nsnap = snL ? (int64_t)snL->n[0] * snL->n[1] * snL->n[2] : sd->n_snap;
    if (nsnap > 0 && snap_out) FGA_TRY(flag_nonfinite(ws, snap_out, nsnap * 6, b->precision, s));
    return FGA_OK;
}

fga_status solve_impl(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd_in, void *seis_out,
                      void *snap_out, cudaStream_t s, double rec_cap, const std::atomic<int> *cancel) {
    fga_stream_t s_ = (fga_stream_t)s;
    FGA_CHECK(m && init && sd_in, "fga_solve: NULL argument");
    // receivers and snapshot points given as (r, theta, phi): Cartesian copies for the rest of the solve
    fga_solve_desc sdc;
    ScopedDevBuf rx_cart, snap_cart;
    FGA_TRY(cartesian_desc(sd_in, sdc, rx_cart, snap_cart, s));
    const fga_solve_desc *sd = &sdc;
    FGA_CHECK(sd->nsteps >= 1 && std::isfinite(sd->dt) && sd->dt != 0.0, "fga_solve: nsteps >= 1 and dt != 0");
    FGA_CHECK(sd->n_times >= 0 && sd->n_rx >= 0 && sd->n_snap >= 0, "fga_solve: negative counts");
    FGA_CHECK(sd->n_times == 0 || sd->times, "fga_solve: times is NULL");
    const fga_lattice *rxL = sd->rx_lattice, *snL = sd->snap_lattice;
    if (rxL) FGA_TRY(check_lattice(rxL, "fga_solve (receivers)"));
    if (snL) FGA_TRY(check_lattice(snL, "fga_solve (snapshot)"));
    FGA_CHECK(rxL || sd->n_rx == 0 || sd->n_times == 0 || (sd->rx && seis_out), "fga_solve: receivers/output missing");
    FGA_CHECK(!rxL || sd->n_times == 0 || seis_out, "fga_solve: seismogram output missing");
    FGA_CHECK(snL || sd->n_snap == 0 || (sd->snap && snap_out), "fga_solve: snapshot points/output missing");
    FGA_CHECK(!snL || snap_out, "fga_solve: snapshot output missing");
    const double T = sd->dt * sd->nsteps;
    std::vector<int> sstep((size_t)sd->n_times);
    std::vector<double> sth((size_t)sd->n_times);
    for (int j = 0; j < sd->n_times; j++) {
        const double t = sd->times[j];
        const bool inside = sd->dt > 0 ? (t > 0 && t <= T * (1 + 1e-12)) : (t < 0 && t >= T * (1 + 1e-12));
        FGA_CHECK(std::isfinite(t) && inside, "fga_solve: sample times must lie in (0, nsteps*dt]");
        FGA_CHECK(j == 0 || (sd->dt > 0 ? t > sd->times[j - 1] : t < sd->times[j - 1]), "fga_solve: times must be monotone");
        const double u = t / sd->dt;
        int n = (int)std::floor(u);
        n = std::min(n, sd->nsteps - 1);
        sstep[(size_t)j] = n;
        sth[(size_t)j] = u - n;
    }
    fga_beams *b = nullptr;
    {
        NvtxRange nr("fga_solve: decompose");
        FGA_TRY(fga_decompose(m, init, &b, s_));
    }
    struct Guard {
        fga_beams *b;
        ~Guard() { fga_beams_destroy(b); }
    } guard{b};
    const double rw = sd->rw > 0 ? sd->rw : 6.0 / std::sqrt(b->k);
    const bool fp64 = b->precision == FGA_PREC_FP64;
    const size_t rb = fp64 ? 8 : 4;
    Workspace &ws = b->ws;
    FGA_TRY(status_reset(ws, s));
    std::vector<double> rxh, snh;
    const bool seis = (rxL || sd->n_rx > 0) && sd->n_times > 0;
    const int64_t nrx = rxL ? (int64_t)rxL->n[0] * rxL->n[1] * rxL->n[2] : sd->n_rx;
    if (seis) {
        if (rxL)
            rxh = lattice_corners(rxL);
        else
            FGA_TRY(host_points(sd->rx, sd->n_rx, rxh, s));
    }
    if (!snL && sd->n_snap > 0) FGA_TRY(host_points(sd->snap, sd->n_snap, snh, s));
    // windows of W steps: the beams are sorted by cell once per window, with cells enlarged by the
    // largest distance a beam can travel inside the window
    const double cmax = std::max(m->cmax[0], m->cmax[1]);
    int W = (int)std::floor(0.25 * rw / std::max(cmax * std::fabs(sd->dt), 1e-300));
    W = std::max(1, std::min(W, 32));
    const double margin = sample_hermite_margin(cmax, sd->dt, W);
    BinGrid grx{};
    if (seis) grx = make_grid(rxh.data(), (int64_t)rxh.size() / 3, rw + margin);
    DevBuf samp;  // per-window sample fractions (R, at offset 0) and local steps (int, at soff)
    HostBuf hsamp;
    const int maxs = sd->n_times;
    const size_t soff = (rb * (size_t)maxs + 15) / 16 * 16;
    const size_t sbytes = soff + sizeof(int) * (size_t)maxs + 16;
    if (maxs > 0) {
        FGA_TRY(samp.ensure(sbytes));
        FGA_TRY(hsamp.ensure(sbytes));
    }
    struct Free {
        DevBuf &d;
        HostBuf &h;
        ~Free() {
            d.release();
            h.release();
        }
    } fr{samp, hsamp};
    if (b->layered) {
        // layered media: samples sit on step ends (every step may split beams at interfaces), and the
        // sums at a sample are taken from the state after that step
        std::vector<int> at((size_t)sd->n_times);
        for (int j = 0; j < sd->n_times; j++) {
            const double u = sd->times[j] / sd->dt;
            const int n = (int)std::lround(u);
            FGA_CHECK(std::fabs(u - n) <= 1e-9 * std::max(1.0, std::fabs(u)) && n >= 1,
                      "fga_solve: in a layered medium the sample times must be whole steps");
            at[(size_t)j] = n;
        }
        int js = 0;
        for (int n = 1; n <= sd->nsteps; n++) {
            if (cancel && cancel->load()) return cancelled(s);
            FGA_TRY(launch_layered_steps(m, b, sd->dt, 1, s));
            if (!seis || js >= sd->n_times || at[(size_t)js] != n) continue;
            FGA_TRY(sync_layered_count(b, s));
            while (js < sd->n_times && at[(size_t)js] == n) {
                void *out = static_cast<char *>(seis_out) + rb * 6 * (size_t)nrx * (size_t)js;
                if (rxL)
                    FGA_TRY(reconstruct_lattice_now(b, rxL, rw, out, s));
                else
                    FGA_TRY(reconstruct_now(b, sd->rx, rxh, sd->n_rx, rw, out, s));
                js++;
            }
        }
        FGA_TRY(sync_layered_count(b, s));
        if (snL)
            FGA_TRY(reconstruct_lattice_now(b, snL, rw, snap_out, s));
        else if (sd->n_snap > 0)
            FGA_TRY(reconstruct_now(b, sd->snap, snh, sd->n_snap, rw, snap_out, s));
        FGA_TRY(flag_solve_nonfinite(b, sd, nrx, seis, seis_out, snap_out, s));
        return status_check(ws, s, "fga_solve");   // synchronises s before the beam set is freed
    }
    // records of one window live in one buffer; cap its size
    size_t free_b = 0, total_b = 0;
    FGA_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double rec_budget = std::min(rec_cap, 0.4 * (double)free_b);
    int js = 0;
    for (int n0 = 0; n0 < sd->nsteps;) {
        if (cancel && cancel->load()) return cancelled(s);
        int nw = std::min(W, sd->nsteps - n0);
        int j1 = js;
        while (seis && j1 < sd->n_times && sstep[(size_t)j1] < n0 + nw) j1++;
        if (j1 == js) {
            FGA_TRY(launch_propagate(m, b, sd->dt, nw, nullptr, s));
            n0 += nw;
            continue;
        }
        NvtxRange nr_win("fga_solve: window");
        int32_t *perm = nullptr;
        {
            NvtxRange nr("fga_solve: binning");
            FGA_TRY(bin_beams(b, grx, &perm, s));
            FGA_TRY(permute_beams(b, perm, s));
        }
        SumPlan plan;
        LatticePlan lplan;
        if (rxL) {
            FGA_TRY(build_lattice_plan(ws, grx, ws.cell_start.as<int32_t>(), *rxL, s, lplan, !fp64, b->k, rw));  // syncs
            for (int c = 0; c < 4; c++) {
                plan.n_in[c] = lplan.n_in[c];
                plan.rec_off[c] = lplan.rec_off[c];
            }
            plan.n_rec = lplan.n_rec;
        } else {
            FGA_TRY(build_sum_plan(ws, grx, ws.cell_start.as<int32_t>(), 4, rxh.data(), sd->n_rx, s, plan));  // syncs
        }
        // shorten the window so that its samples' records fit the budget (a shorter window keeps the
        // cell margin valid)
        const int64_t per_sample = (int64_t)rb * REC * std::max<int64_t>(plan.n_rec, 1);
        const int smax = (int)std::max<double>(1.0, std::floor(rec_budget / (double)per_sample));
        if (j1 - js > smax) {
            j1 = js + smax;
            nw = sstep[(size_t)(j1 - 1)] - n0 + 1;  // end the window with the step of its last sample
            while (j1 < sd->n_times && sstep[(size_t)j1] < n0 + nw) j1++;
        }
        const int ns = j1 - js;
        char *hth = hsamp.as<char>();
        int *hs = reinterpret_cast<int *>(hth + soff);
        for (int j = 0; j < ns; j++) {
            hs[j] = sstep[(size_t)(js + j)] - n0;
            if (fp64)
                reinterpret_cast<double *>(hth)[j] = sth[(size_t)(js + j)];
            else
                reinterpret_cast<float *>(hth)[j] = (float)sth[(size_t)(js + j)];
        }
        FGA_CUDA(cudaMemcpyAsync(samp.p, hsamp.p, sbytes, cudaMemcpyHostToDevice, s));
        FGA_TRY(ws.rec.ensure((size_t)per_sample * ns));
        // FP32 lattice sums take their operand scale from the amplitude bound the RK4 kernel forms per sample
        unsigned *amax = nullptr;
        if (rxL && !fp64) {
            FGA_TRY(ws.rec_amax.ensure(sizeof(unsigned) * (size_t)ns));
            amax = ws.rec_amax.as<unsigned>();
            FGA_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned) * (size_t)ns, s));
        }
        SampleWindow sw{ns, reinterpret_cast<const int *>(samp.as<char>() + soff), samp.p, ws.rec.p, {}, {}, plan.n_rec,
                        amax};
        for (int c = 0; c < 4; c++) {
            sw.n_in[c] = plan.n_in[c];
            sw.rec_off[c] = plan.rec_off[c];
        }
        {
            NvtxRange nr("fga_solve: propagate");
            FGA_TRY(launch_propagate(m, b, sd->dt, nw, &sw, s));
        }
        NvtxRange nr_sums("fga_solve: sums");
        for (int j = 0; j < ns; j++) {
            void *out = static_cast<char *>(seis_out) + rb * 6 * (size_t)nrx * (size_t)(js + j);
            const void *rec = static_cast<const char *>(ws.rec.p) + (size_t)per_sample * j;
            if (rxL)
                FGA_TRY(run_lattice(ws, lplan, b->precision, rec, b->k, rw, out, s, P_GATHER,
                                    amax ? reinterpret_cast<const float *>(amax + j) : nullptr));
            else
                FGA_TRY(run_sum(ws, plan, b->precision, rec, sd->rx, b->k, rw, out, s));
        }
        js = j1;
        n0 += nw;
    }
    {
        NvtxRange nr("fga_solve: snapshot");
        if (snL)
            FGA_TRY(reconstruct_lattice_now(b, snL, rw, snap_out, s));
        else if (sd->n_snap > 0)
            FGA_TRY(reconstruct_now(b, sd->snap, snh, sd->n_snap, rw, snap_out, s));
    }
    FGA_TRY(flag_solve_nonfinite(b, sd, nrx, seis, seis_out, snap_out, s));
    // the beam set is freed by the guard; its buffers must not be in use (the check synchronises s)
    return status_check(ws, s, "fga_solve");
}
}  // namespace fga

extern "C" {

fga_status fga_beams_count(const fga_beams *b, int64_t *n_by_class) {
    FGA_CHECK(b && n_by_class, "fga_beams_count: NULL argument");
    if (!b->layered) {
        for (int c = 0; c < 4; c++) n_by_class[c] = b->n_cls[c];
        return FGA_OK;
    }
    FGA_TRY(sync_layered_count(const_cast<fga_beams *>(b), b->last_stream));
    std::vector<int32_t> fl((size_t)b->nb);
    if (b->nb > 0) FGA_CUDA(cudaMemcpy(fl.data(), b->flags.p, 4 * (size_t)b->nb, cudaMemcpyDeviceToHost));
    for (int c = 0; c < 4; c++) n_by_class[c] = 0;
    for (int32_t f : fl)
        if (!(f & FL_DEAD)) n_by_class[f & FL_CLASS_MASK]++;
    return FGA_OK;
}

// the stored state (all NFS fields) of the first nb slots as float64, field-major with stride cap
static fga_status state_to_host(const fga_beams *b, int64_t cap, std::vector<double> &st) {
    st.resize((size_t)(NFS * cap));
    if (b->precision == FGA_PREC_FP64) {
        FGA_CUDA(cudaMemcpy(st.data(), b->state.p, 8 * (size_t)(NFS * cap), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> sf((size_t)(NFS * cap));
        FGA_CUDA(cudaMemcpy(sf.data(), b->state.p, 4 * (size_t)(NFS * cap), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < sf.size(); i++) st[i] = sf[i];
    }
    return FGA_OK;
}
// one exported row: the 46 state values with Q's compensation folded in, then two zeros
static void export_row(const std::vector<double> &st, int64_t cap, int64_t i, double *o) {
    for (int f = 0; f < NF; f++) o[f] = st[(size_t)(f * cap + i)];
    for (int d = 0; d < 3; d++) o[F_Q + d] -= st[(size_t)((F_QC + d) * cap + i)];
    o[46] = 0.0;
    o[47] = 0.0;
}

// S polarisation frame of P (host): N_sh = e x P / |e x P| (e = e3, or e1 when ref_e1), N_sv = N_sh x P/|P|
static void s_frame_host(const double *P, bool ref_e1, double *Nsv, double *Nsh) {
    const double v[3] = {ref_e1 ? 0.0 : -P[1], ref_e1 ? -P[2] : P[0], ref_e1 ? P[1] : 0.0};
    const double vn = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double pn = std::sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    for (int c = 0; c < 3; c++) Nsh[c] = v[c] / vn;
    Nsv[0] = (Nsh[1] * P[2] - Nsh[2] * P[1]) / pn;
    Nsv[1] = (Nsh[2] * P[0] - Nsh[0] * P[2]) / pn;
    Nsv[2] = (Nsh[0] * P[1] - Nsh[1] * P[0]) / pn;
}

// an exported row of a tilted layered set, from the layer frame back to global coordinates: Q, P and the
// rows of dzQ, dzP by R^T; an S beam's polarisation vector re-expressed in the S frame of the global P
// (its frame bit in *mt chosen by the same rule as at decomposition)
static void row_to_global(const double *Rm, double *o, int32_t *mt) {
    auto rotT = [&](double *v) {
        double w[3];
        for (int c = 0; c < 3; c++) w[c] = Rm[c] * v[0] + Rm[3 + c] * v[1] + Rm[6 + c] * v[2];
        for (int c = 0; c < 3; c++) v[c] = w[c];
    };
    double Pl[3] = {o[F_P], o[F_P + 1], o[F_P + 2]};
    rotT(o + F_Q);
    rotT(o + F_P);
    for (int base : {F_DQ, F_DP})
        for (int m = 0; m < 3; m++)
            for (int part = 0; part < 2; part++) {
                double v[3];
                for (int j = 0; j < 3; j++) v[j] = o[base + 2 * (3 * m + j) + part];
                rotT(v);
                for (int j = 0; j < 3; j++) o[base + 2 * (3 * m + j) + part] = v[j];
            }
    if ((*mt & FL_CLASS_MASK) >= 2) {
        double Nsv[3], Nsh[3], Ar[3], Ai[3];
        s_frame_host(Pl, (*mt & FL_REF_E1) != 0, Nsv, Nsh);
        for (int c = 0; c < 3; c++) {
            Ar[c] = o[F_A0] * Nsv[c] + o[F_A1] * Nsh[c];
            Ai[c] = o[F_A0 + 1] * Nsv[c] + o[F_A1 + 1] * Nsh[c];
        }
        rotT(Ar);
        rotT(Ai);
        const double *P = o + F_P;
        const bool r1 = (P[0] * P[0] + P[1] * P[1]) < 0.01 * (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
        *mt = r1 ? (*mt | FL_REF_E1) : (*mt & ~FL_REF_E1);
        s_frame_host(P, r1, Nsv, Nsh);
        o[F_A0] = Ar[0] * Nsv[0] + Ar[1] * Nsv[1] + Ar[2] * Nsv[2];
        o[F_A0 + 1] = Ai[0] * Nsv[0] + Ai[1] * Nsv[1] + Ai[2] * Nsv[2];
        o[F_A1] = Ar[0] * Nsh[0] + Ar[1] * Nsh[1] + Ar[2] * Nsh[2];
        o[F_A1 + 1] = Ai[0] * Nsh[0] + Ai[1] * Nsh[1] + Ai[2] * Nsh[2];
    }
}

fga_status fga_beams_export_all(const fga_beams *b, int64_t cap, int64_t *n_out, int64_t *dropped, double *state,
                                int32_t *meta, int64_t *mesh_id, int64_t *path) {
    FGA_CHECK(b && n_out && cap >= 0, "fga_beams_export_all: NULL argument or negative cap");
    FGA_CUDA(cudaStreamSynchronize(b->last_stream));
    FGA_TRY(sync_layered_count(const_cast<fga_beams *>(b), b->last_stream));
    const int64_t nb = b->nb, scap = b->cap;
    std::vector<int32_t> ids((size_t)nb), fl((size_t)nb);
    std::vector<long long> pa((size_t)nb, 0);
    if (nb > 0) {
        FGA_CUDA(cudaMemcpy(ids.data(), b->id.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost));
        FGA_CUDA(cudaMemcpy(fl.data(), b->flags.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost));
        if (b->layered) FGA_CUDA(cudaMemcpy(pa.data(), b->path.p, 8 * (size_t)nb, cudaMemcpyDeviceToHost));
    }
    std::vector<double> st;
    if (state && nb > 0) FGA_TRY(state_to_host(b, scap, st));
    int64_t k = 0;
    for (int64_t i = 0; i < nb; i++) {
        if (fl[(size_t)i] & FL_DEAD) continue;
        if (k < cap) {
            if (meta) meta[k] = fl[(size_t)i];
            if (mesh_id) mesh_id[k] = ids[(size_t)i];
            if (path) path[k] = pa[(size_t)i];
            if (state) {
                export_row(st, scap, i, state + k * 48);
                if (b->tilted) {
                    int32_t mt = fl[(size_t)i];
                    row_to_global(b->R, state + k * 48, &mt);
                    if (meta) meta[k] = mt;
                }
            }
        }
        k++;
    }
    *n_out = k;
    if (dropped) {
        unsigned long long c[2] = {0, 0};
        if (b->layered) FGA_CUDA(cudaMemcpy(c, b->counts.p, sizeof c, cudaMemcpyDeviceToHost));
        *dropped = (int64_t)c[1];
    }
    return FGA_OK;
}

fga_status fga_beams_export(const fga_beams *b, double *state_host, int32_t *meta_host) {
    FGA_CHECK(b, "fga_beams_export: NULL beams");
    if (b->layered) {
        set_error("fga_beams_export: beams of a layered medium split at interfaces; use fga_beams_export_all");
        return FGA_ERR_UNSUPPORTED;
    }
    FGA_CUDA(cudaStreamSynchronize(b->last_stream));
    const int64_t cap = b->cap, nb = b->nb;
    std::vector<int32_t> ids((size_t)nb), fl((size_t)nb);
    if (nb > 0) {
        FGA_CUDA(cudaMemcpy(ids.data(), b->id.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost));
        FGA_CUDA(cudaMemcpy(fl.data(), b->flags.p, 4 * (size_t)nb, cudaMemcpyDeviceToHost));
    }
    std::vector<double> st;
    if (state_host && nb > 0) FGA_TRY(state_to_host(b, cap, st));
    // mesh order per class: class blocks in class order, beams by mesh index within a block (a
    // selection keeps a subset of the mesh points, so the row is the beam's rank, not its index)
    std::vector<int64_t> order((size_t)nb);
    for (int64_t i = 0; i < nb; i++) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t c) {
        const int ca = fl[(size_t)a] & FL_CLASS_MASK, cc = fl[(size_t)c] & FL_CLASS_MASK;
        return ca != cc ? ca < cc : ids[(size_t)a] < ids[(size_t)c];
    });
    for (int64_t row = 0; row < nb; row++) {
        const int64_t i = order[(size_t)row];
        if (meta_host) meta_host[row] = fl[(size_t)i];
        if (state_host) export_row(st, cap, i, state_host + row * 48);
    }
    return FGA_OK;
}

fga_status fga_beams_params(const fga_beams *b, double *k, double *w, int *precision) {
    FGA_CHECK(b, "fga_beams_params: NULL beams");
    if (k) *k = b->k;
    if (w) *w = b->w;
    if (precision) *precision = b->precision;
    return FGA_OK;
}

fga_status fga_beams_import(int64_t n, const double *state, const int32_t *meta, double k, double w, int precision,
                            fga_beams **out, fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(out && (n == 0 || (state && meta)), "fga_beams_import: NULL argument");
    FGA_CHECK(n >= 0 && n < ((int64_t)1 << 31), "fga_beams_import: n must lie in [0, 2^31)");
    FGA_CHECK(std::isfinite(k) && k > 0 && std::isfinite(w) && w > 0, "fga_beams_import: k and w must be > 0");
    FGA_CHECK(precision == FGA_PREC_FP32 || precision == FGA_PREC_FP64, "fga_beams_import: bad precision");
    for (int64_t i = 0; i < n; i++)
        FGA_CHECK((meta[i] & ~(FL_CLASS_MASK | FL_REF_E1)) == 0, "fga_beams_import: meta holds more than class and frame bits");
    fga_beams *b = new fga_beams();
    std::unique_ptr<fga_beams, fga_status (*)(fga_beams *)> hold(b, fga_beams_destroy);
    b->precision = precision;
    b->k = k;
    b->w = w;
    // class blocks in class order, beams in their given order within a block
    std::vector<int64_t> order((size_t)n);
    int64_t cnt[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) cnt[meta[i] & FL_CLASS_MASK]++;
    int64_t off = 0;
    for (int c = 0; c < 4; c++) {
        b->off_cls[c] = off;
        b->n_cls[c] = cnt[c];
        off += cnt[c];
    }
    b->nb = n;
    b->cap = std::max<int64_t>(32, (n + 31) / 32 * 32);
    int64_t pos[4] = {b->off_cls[0], b->off_cls[1], b->off_cls[2], b->off_cls[3]};
    for (int64_t i = 0; i < n; i++) order[(size_t)pos[meta[i] & FL_CLASS_MASK]++] = i;
    const size_t rb = precision == FGA_PREC_FP64 ? 8 : 4;
    FGA_TRY(b->state.ensure(rb * NFS * b->cap));
    FGA_TRY(b->flags.ensure(4 * b->cap));
    FGA_TRY(b->id.ensure(4 * b->cap));
    // structure of arrays on the host, then one copy each (compensation of Q starts at zero)
    std::vector<int32_t> fl((size_t)b->cap, 0), ids((size_t)b->cap, 0);
    std::vector<double> sd((size_t)(NFS * b->cap), 0.0);
    for (int64_t r = 0; r < n; r++) {
        const int64_t i = order[(size_t)r];
        for (int f = 0; f < NF; f++) sd[(size_t)(f * b->cap + r)] = state[i * 48 + f];
        fl[(size_t)r] = meta[i];
        ids[(size_t)r] = (int32_t)(r - b->off_cls[meta[i] & FL_CLASS_MASK]);
    }
    if (precision == FGA_PREC_FP64) {
        FGA_CUDA(cudaMemcpy(b->state.p, sd.data(), 8 * sd.size(), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> sf(sd.size());
        for (size_t i = 0; i < sd.size(); i++) sf[i] = (float)sd[i];
        FGA_CUDA(cudaMemcpy(b->state.p, sf.data(), 4 * sf.size(), cudaMemcpyHostToDevice));
    }
    FGA_CUDA(cudaMemcpy(b->flags.p, fl.data(), 4 * fl.size(), cudaMemcpyHostToDevice));
    FGA_CUDA(cudaMemcpy(b->id.p, ids.data(), 4 * ids.size(), cudaMemcpyHostToDevice));
    b->last_stream = s;
    *out = hold.release();
    return FGA_OK;
}

fga_status fga_beams_destroy(fga_beams *b) {
    if (!b) return FGA_OK;
    b->ws.release();
    for (DevBuf *d : {&b->state, &b->state_alt, &b->flags, &b->flags_alt, &b->id, &b->id_alt, &b->path, &b->counts,
                      &b->n_begin})
        d->release();
    delete b;
    return FGA_OK;
}

fga_status fga_profile_enable(int mode) {
    FGA_CHECK(mode >= 0 && mode <= 3, "fga_profile_enable: mode must be 0, 1, 2 or 3");
    g_prof.mode = mode;
    return FGA_OK;
}

fga_status fga_profile_read(fga_profile_t *out, int reset) {
    FGA_CHECK(out, "fga_profile_read: NULL argument");
    g_prof.fold();
    std::memset(out, 0, sizeof *out);
    out->launches = g_prof.launches;
    for (int c = 0; c < P_NCAT; c++) {
        out->count[c] = g_prof.count[c];
        out->ms[c] = g_prof.ms[c];
    }
    out->beam_steps = g_prof.beam_steps;
    out->pairs_tested = g_prof.pairs_tested;
    out->pairs_in_window =
        read_pair_counter(reset != 0) + read_lattice_pair_counter(reset != 0) + read_tc_pair_counter(reset != 0) +
        read_plane_pair_counter(reset != 0);
    if (reset) {
        g_prof.launches = g_prof.beam_steps = g_prof.pairs_tested = 0;
        for (int c = 0; c < P_NCAT; c++) {
            g_prof.count[c] = 0;
            g_prof.ms[c] = 0.0;
        }
    }
    return FGA_OK;
}

fga_status fga_bin(const float *Q, int64_t n, const float origin[3], float inv_h, const int nc[3], int32_t *keys,
                   int32_t *perm, int32_t *cell_start, fga_stream_t s_) {
    cudaStream_t s = (cudaStream_t)s_;
    FGA_CHECK(origin && nc && perm && cell_start, "fga_bin: NULL argument");
    FGA_CHECK(n >= 0 && n < ((int64_t)1 << 31), "fga_bin: n out of range");
    FGA_CHECK(n == 0 || Q, "fga_bin: NULL centres");
    FGA_CHECK(std::isfinite(inv_h) && inv_h > 0, "fga_bin: inv_h must be > 0");
    BinGrid g{};
    int64_t ncell = 1;
    for (int d = 0; d < 3; d++) {
        FGA_CHECK(nc[d] >= 1, "fga_bin: nc must be >= 1");
        g.o[d] = origin[d];
        g.nc[d] = nc[d];
        ncell *= nc[d];
    }
    FGA_CHECK(ncell < (1 << 24), "fga_bin: too many cells");
    g.ncells = (int)ncell;
    g.inv_h = inv_h;
    g.clamp = true;
    static thread_local Workspace ws;  // scratch of the standalone binning entry point
    FGA_TRY(ws.keys.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
    FGA_TRY(bin_centres(g, Q, Q_F32_AOS3, 0, n, nullptr, ws.keys.as<int32_t>(), s));
    if (keys && n > 0) FGA_CUDA(cudaMemcpyAsync(keys, ws.keys.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    int32_t *pv = nullptr;
    FGA_TRY(sort_keys_to_perm(ws, ws.keys.as<int32_t>(), n, g.ncells, &pv, cell_start, s));
    if (n > 0) FGA_CUDA(cudaMemcpyAsync(perm, pv, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    FGA_CUDA(cudaStreamSynchronize(s));
    return FGA_OK;
}

}  // extern "C"
