// Internal declarations of the GB300 FGA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fga.h"

namespace fga {

// Beam state: 46 reals per beam, stored structure-of-arrays with stride `cap` (field f of beam b
// at base[f * cap + b]):
//   0-2 Q, 3-5 P, 6-23 dzQ (entry [m][j] re at 6 + 2(3m+j), im at 7 + 2(3m+j)), 24-41 dzP (same
//   order), 42-43 amplitude a (P) or a_sv (S), 44-45 a_sh (S; zero for P).
// Three more stored fields, 46-48, hold the compensation of Q's running sum (Kahan): each step adds
// its increment to Q with the rounding error carried to the next step, so Q = stored Q - compensation
// to far better than one rounding per step (thousands of steps of beams hundreds of wavelengths
// from the origin would otherwise drift by many ulps of |Q|).
constexpr int NF = 46;
constexpr int F_Q = 0, F_P = 3, F_DQ = 6, F_DP = 24, F_A0 = 42, F_A1 = 44;
constexpr int F_QC = NF;       // compensation of Q (3 fields)
constexpr int NFS = NF + 3;    // stored fields per beam

// Q <- Q + inc with the compensation c carried between steps (Kahan summation)
template <typename R> __device__ __forceinline__ void kahan_add(R &q, R &c, R inc) {
    const R yk = inc - c;
    const R t = q + yk;
    c = (t - q) - yk;
    q = t;
}
// Reconstruction record: Q(3), P(3), polarised amplitude times the quadrature weight (3 complex).
constexpr int REC = 12;
constexpr int MAX_LAYERS = 8;

// flags per beam
constexpr int FL_CLASS_MASK = 3;  // 0 P+, 1 P-, 2 S+, 3 S-
constexpr int FL_REF_E1 = 4;      // S frame built on e1 instead of e3
// bits 4-7: layer of the beam (layered media); bits 8-11: interfaces crossed so far
constexpr int FL_DEAD = 1 << 12;  // dropped at an interface (layered media)
constexpr int FL_ROOT_SHIFT = 13; // bits 13-14: class of the initial beam of the lineage (layered media)

struct ModelDev {
    int kind;
    double cp0, cs0, amp, cs_ratio;
    int n[3];
    double o[3], h[3], inv_h[3];
    const float4 *gp, *gs;  // grid: 3 float4 (10 fields + 2 pad) per node
    int nlay;
    double zif[MAX_LAYERS], lcp[MAX_LAYERS], lcs[MAX_LAYERS], lrho[MAX_LAYERS];
    // tilted layers: rows of R are the layer frame's axes in global coordinates (row 2 = the normal);
    // beams live in the layer frame, x' = R x
    int tilted;
    double R[9];
    // spherical layers: the interfaces are |x - ctr| = -zif[i] (zif holds minus the radii, so that the
    // depth -|x - ctr| orders the layers as x3 does for flat ones)
    int shells;
    double ctr[3];
    // undulating layers: interface i is x3 = zif[i] + uamp[i] cos(uk[0] x1) cos(uk[1] x2)
    int undul;
    double uamp[MAX_LAYERS], uk[2];
    // FP32 copies of the scalar parameters: the FP32 kernels read these and never convert from
    // double (FP64 instructions are very slow on this GPU)
    float fcp0, fcs0, famp, fcs_ratio, fo[3], finv_h[3], fzif[MAX_LAYERS], flcp[MAX_LAYERS], flcs[MAX_LAYERS];
    float fuamp[MAX_LAYERS], fuk[2];
    void fill_f32() {
        fcp0 = (float)cp0;
        fcs0 = (float)cs0;
        famp = (float)amp;
        fcs_ratio = (float)cs_ratio;
        for (int d = 0; d < 3; d++) {
            fo[d] = (float)o[d];
            finv_h[d] = (float)inv_h[d];
        }
        fuk[0] = (float)uk[0];
        fuk[1] = (float)uk[1];
        for (int l = 0; l < MAX_LAYERS; l++) {
            fuamp[l] = (float)uamp[l];
            fzif[l] = (float)zif[l];
            flcp[l] = (float)lcp[l];
            flcs[l] = (float)lcs[l];
        }
    }
};

// An orthonormal frame whose third axis is the unit vector n, as the rows of R (x' = R x): the first
// axis is the normalised cross product of the coordinate axis least parallel to n with n, the second
// completes the right-handed frame.
__host__ __device__ inline void frame_from_normal(const double n[3], double R[9]) {
    const double a0 = fabs(n[0]), a1 = fabs(n[1]), a2 = fabs(n[2]);
    const int ax = (a0 <= a1 && a0 <= a2) ? 0 : (a1 <= a2 ? 1 : 2);
    double a[3] = {0.0, 0.0, 0.0}, e1[3];
    a[ax] = 1.0;
    e1[0] = a[1] * n[2] - a[2] * n[1];
    e1[1] = a[2] * n[0] - a[0] * n[2];
    e1[2] = a[0] * n[1] - a[1] * n[0];
    const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int c = 0; c < 3; c++) e1[c] /= l1;
    R[0] = e1[0];
    R[1] = e1[1];
    R[2] = e1[2];
    R[3] = n[1] * e1[2] - n[2] * e1[1];
    R[4] = n[2] * e1[0] - n[0] * e1[2];
    R[5] = n[0] * e1[1] - n[1] * e1[0];
    R[6] = n[0];
    R[7] = n[1];
    R[8] = n[2];
}

// error handling ---------------------------------------------------------------------------
void set_error(const std::string &msg);
fga_status cuda_fail(cudaError_t e, const char *what);

#define FGA_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ::fga::cuda_fail(e_, #call); \
    } while (0)
#define FGA_CHECK(cond, msg)                 \
    do {                                     \
        if (!(cond)) {                       \
            ::fga::set_error(msg);           \
            return FGA_ERR_INVALID_ARG;      \
        }                                    \
    } while (0)
#define FGA_TRY(call)                  \
    do {                               \
        fga_status fga_st_ = (call);   \
        if (fga_st_ != FGA_OK) return fga_st_; \
    } while (0)

// profiling: launch counters and CUDA-event device times per kernel category -------------------
// P_GATHER: Gaussian sums at sample times inside a solve; P_GATHER_STATE: sums at the current state
// (snapshots, fga_reconstruct*)
enum ProfCat {
    P_DECOMP = 0,
    P_PROP = 1,
    P_BIN = 2,
    P_REC = 3,
    P_GATHER = 4,
    P_REDUCE = 5,
    P_GATHER_STATE = 6,
    P_OTHER_LAYER = 7,
    P_ADJ_FWD = 8,   // adjoint: forward recomputation (checkpoints, segments)
    P_ADJ_REV = 9,   // adjoint: reverse steps
    P_ADJ_INIT = 10, // adjoint: initial-amplitude term
    P_MISFIT = 11,   // traveltime misfit and adjoint source
    P_NCAT = 12
};
struct ProfScope {  // wraps one kernel launch on stream s
    ProfScope(int cat, cudaStream_t s);
    ~ProfScope();
    int idx;
    cudaStream_t s;
};
// NVTX range around a phase of a call (decomposition, a window's propagation or sums, a snapshot, the
// adjoint's passes): visible in Nsight timelines, a single branch when no tool is attached
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
bool prof_counting();
void prof_add_beam_steps(int64_t n);
void prof_add_pairs_tested(int64_t n);
int64_t read_pair_counter(bool reset);  // gather.cu

// grow-only device / pinned-host buffers -----------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    fga_status ensure(size_t need);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};
// a DevBuf owned by one scope (function-local scratch): released when the scope ends, also on early returns
struct ScopedDevBuf : DevBuf {
    ScopedDevBuf() = default;
    ScopedDevBuf(const ScopedDevBuf &) = delete;
    ScopedDevBuf &operator=(const ScopedDevBuf &) = delete;
    ~ScopedDevBuf() { release(); }
};
struct HostBuf {
    void *p = nullptr;
    size_t bytes = 0;
    fga_status ensure(size_t need);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// per-thread block cache for DevBuf/HostBuf (see api.cu); s: the one stream the thread uses
void block_cache_enable(cudaStream_t s);
void block_cache_disable();
void block_cache_trim(size_t keep_bytes);
size_t block_cache_bytes();

// scratch used by binning and the Gaussian sum
struct Workspace {
    DevBuf keys, keys_alt, vals, vals_alt, hist, scan_blocks, cell_start, rec, items, tiles, partial, pts;
    DevBuf rec_amax;   // per sample of a window: bound of the records' amplitude entries (FP32 path)
    // status words of one call: [0] a bounded wait of the tensor-core lattice sum ran out,
    // [1] non-finite values in the beam state or the outputs
    DevBuf status;
    HostBuf h_cell_start, h_items, h_tiles;
    void release();
};

}  // namespace fga

struct fga_model {
    fga::ModelDev dev;
    fga::DevBuf grid;
    double cmax[2];  // largest P and S speed of the medium (bounds beam displacement)
};

struct fga_beams {
    int precision;
    double k, w;
    // tilted layered media: the state is in the layer frame x' = R x (R as in ModelDev)
    bool tilted = false;
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    int64_t nb, cap;
    int64_t n_cls[4], off_cls[4];
    fga::DevBuf state, state_alt, flags, flags_alt, id, id_alt;
    mutable fga::Workspace ws;
    cudaStream_t last_stream = nullptr;
    // layered media: the population grows at interfaces (slots [0, counts[0]) used, capacity cap)
    bool layered = false;
    int gmax = 4;            // a beam is dropped at its (gmax+1)-th interface
    double rel_min = 1e-6;   // children below rel_min of the incident amplitude are not created
    fga::DevBuf path, counts, n_begin;  // lineage (parent*4 + child slot + 1); [slots used, overflow]
};

namespace fga {

// kernels and launchers (one per translation unit area) ------------------------------------
// tc_gemm.cu: complex GEMM C[z][m][n] = scale sum_k A[z][m][k] B[n][k] on the tensor cores (FP16 split,
// FP32 accumulation); |B| <= 1; |Re|, |Im| of A bounded by (*amax) * amax_factor; *err set if a wait ran out
template <typename TA>
fga_status tc_cgemm(const TA *A, int64_t sAz, int64_t sAm, int64_t sAk, const float2 *B, int64_t sBn, int64_t sBk,
                    float2 *C, int64_t sCz, int64_t sCm, int64_t sCn, int Z, int64_t M, int N, int K, float scale,
                    const float *amax, float amax_factor, int *err, cudaStream_t s);
fga_status tc_absmax(const double2 *x, int64_t n, float *out, cudaStream_t s);
// decompose.cu
fga_status decompose_impl(const fga_model *m, const fga_init_desc *d, fga_beams **out, cudaStream_t s);
fga_status transform_impl(const fga_init_desc *d, void *F_out, cudaStream_t s);
// propagate.cu
struct SampleWindow {
    int n;                  // samples in this window
    const int *step;        // DEVICE: local step of each sample (0-based within the window)
    const void *theta;      // DEVICE: R fraction in [0,1]
    void *rec;              // DEVICE: records [n][n_rec][REC]
    int64_t n_in[4];        // class c: the first n_in[c] beams of its block get records ...
    int64_t rec_off[4];     // ... at record index rec_off[c] + (position - off_cls[c])
    int64_t n_rec;          // records per sample
    unsigned *amax;         // DEVICE, FP32 path or NULL: per sample, bits of max |A entry| over its records
};
fga_status launch_propagate(const fga_model *m, fga_beams *b, double dt, int nsteps, const SampleWindow *sw,
                            cudaStream_t s);
// records of the current state for the first n_in[c] sorted beams of class c, which start at sorted
// position beg[c] (perm: sorted position -> beam), written at rec_off[c] + (position - beg[c])
fga_status launch_records_from_state(const fga_beams *b, const int32_t *perm, const int64_t beg[4],
                                     const int64_t n_in[4], const int64_t rec_off[4], void *rec, cudaStream_t s);
// api.cu: points (r, theta, phi) -> Cartesian device copies (Sec. 3); a solve descriptor with its spherical
// point arrays replaced by Cartesian copies held in rx / snap
fga_status spherical_points(const double *rtp, int64_t n, DevBuf &out, cudaStream_t s);
fga_status cartesian_desc(const fga_solve_desc *sd, fga_solve_desc &out, DevBuf &rx, DevBuf &snap, cudaStream_t s);
// api.cu: the whole forward solve (fga_solve) with a cap on the record buffer of one window
fga_status solve_impl(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd, void *seis_out,
                      void *snap_out, cudaStream_t s, double rec_cap, const std::atomic<int> *cancel);
// layered.cu
fga_status launch_layered_steps(const fga_model *m, fga_beams *b, double dt, int nsteps, cudaStream_t s);
// layered media: refresh b->nb from the device slot counter (synchronises s)
fga_status sync_layered_count(fga_beams *b, cudaStream_t s);
// gather.cu
struct BinGrid {
    float o[3];
    float inv_h;
    int nc[3];
    int ncells;       // nc0*nc1*nc2
    bool clamp;       // true: clamp keys into the grid; false: out-of-grid centres go to bucket ncells
};
// exclusive prefix sum of n uint32 in place on stream s (synchronises s before returning)
fga_status scan_exclusive_u32(uint32_t *a, int64_t n, cudaStream_t s);
fga_status bin_centres(const BinGrid &g, const void *Q_src, int q_kind, int64_t q_stride, int64_t n,
                       const int32_t *cls_or_null, int32_t *keys, cudaStream_t s);
fga_status radix_sort_pairs(Workspace &ws, int32_t *keys, int32_t *vals, int64_t n, int bits,
                            int32_t **keys_out, int32_t **vals_out, cudaStream_t s);
fga_status cell_starts(const int32_t *sorted_keys, int64_t n, int nbuckets, int32_t *cell_start, cudaStream_t s);
fga_status permute_beams(fga_beams *b, const int32_t *perm, cudaStream_t s);
// binning grid covering every point of a set, expanded by `reach`, with cells >= reach
BinGrid make_grid(const double *pts_host, int64_t n, double reach);

}  // namespace fga
