// Internal interface of binning and the Gaussian sum.
#pragma once

#include "fga_internal.cuh"

namespace fga {

// sources of beam centres for the key kernel
enum { Q_F32_AOS3 = 0, Q_F32_SOA = 1, Q_F64_SOA = 2 };

// Work split of a Gaussian sum at a fixed point set: tiles of 32 points of one cell, items =
// (tile, [begin, end) of the cell-sorted beams), item_start[t] .. item_start[t+1] the items of tile t.
struct SumPlan {
    int ntiles = 0, nitems = 0;
    const int32_t *tile_pts = nullptr;   // DEVICE [ntiles][32] point index or -1
    const int32_t *item_start = nullptr; // DEVICE [ntiles + 1]
    const int4 *items = nullptr;         // DEVICE [nitems] {tile, begin, end, 0}: record indices
    int64_t pairs_tested = 0;            // point x candidate-beam pairs (upper bound of the work)
    // Records are kept only for beams inside the grid: class c's in-grid beams sit at sorted
    // positions off_cls[c] .. off_cls[c] + n_in[c] and get record indices rec_off[c] + (pos - off_cls[c]).
    int64_t n_in[4] = {0, 0, 0, 0}, rec_off[4] = {0, 0, 0, 0}, n_rec = 0, beg[4] = {0, 0, 0, 0};
};

// Work split of a Gaussian sum on a tensor lattice: tiles are T0 x T1 x T2 boxes of the lattice.
struct LatticePlan {
    int T[3] = {1, 1, 1}, n[3] = {0, 0, 0}, nt[3] = {0, 0, 0};
    int ntiles = 0, nitems = 0;
    const double *ax[3] = {nullptr, nullptr, nullptr};  // DEVICE axis coordinates
    const int32_t *item_start = nullptr;
    const int4 *items = nullptr;
    int64_t pairs_tested = 0;
    int64_t n_in[4] = {0, 0, 0, 0}, rec_off[4] = {0, 0, 0, 0}, n_rec = 0, beg[4] = {0, 0, 0, 0};
    // axes with uniform spacing (coordinate i = x0 + i * dx to 1e-12 relative): the tensor-core kernel forms
    // their 1-D factors by recurrence
    bool uniform[3] = {false, false, false};
    double dx[3] = {0, 0, 0};
    double x_first[3] = {0, 0, 0};   // first coordinate of each axis
};
// tc: tile shape and work split of the tensor-core kernel (the FP32 path); else the CUDA-core kernel's
fga_status build_lattice_plan(Workspace &ws, const BinGrid &g, const int32_t *cell_start_dev, const fga_lattice &L,
                              cudaStream_t s, LatticePlan &plan, bool tc, double k, double rw);
// The tensor-core lattice kernels form a beam's 1-D factors exp(i k P (x - Q) - k (x - Q)^2 / 2) along a
// uniform axis by recurrence: the first point directly, then ratios exp(i k P h - k h (x - Q + h/2)),
// each ratio times exp(-k h^2).  In FP32 a first value with k (x - Q)^2 / 2 > 87 underflows and
// zeroes the run; a kept beam lies within rw of the tile, and the values lost that way stay below
// e^-14 of its amplitude when a run spans at most recurrence_span_max(k, rw).  The ratio itself is
// finite while k h (span + rw + h) <= 87 (recurrence_ratio_ok); otherwise the run is one point.
double recurrence_span_max(double k, double rw);
bool recurrence_ratio_ok(double k, double step, double span, double rw);
void tile_shape_tc(const fga_lattice &L, int T[3]);
// single-plane lattices with uniform axes 0 and 1: the warp-specialised plane kernel (tc_plane.cu)
void tile_shape_plane(const fga_lattice &L, int T[3]);
bool plane_tc_eligible(const LatticePlan &plan);
// amax: DEVICE bound of the records' |A| entries (bits of a non-negative float), or NULL to compute it
fga_status run_plane_tc(Workspace &ws, const LatticePlan &plan, const void *rec, double k, double rw, void *u,
                        cudaStream_t s, int cat, const float *amax = nullptr);
int64_t read_plane_pair_counter(bool reset);
// |A| bound of n records into *out (zeroed by the caller)
fga_status rec_absmax(const float *rec, int64_t n, float *out, cudaStream_t s, int cat);
fga_status run_lattice_tc(Workspace &ws, const LatticePlan &plan, const void *rec, double k, double rw, void *u,
                          cudaStream_t s, int cat, const float *amax = nullptr);
fga_status lattice_reduce_f32(const float *partial, const LatticePlan &plan, void *u, cudaStream_t s);
int64_t read_tc_pair_counter(bool reset);
// per-beam-set status words (Workspace::status): zeroed by status_reset before a call's work, read by
// status_check after it (synchronises s): a tensor-core wait that ran out gives FGA_ERR_TIMEOUT,
// non-finite values FGA_ERR_NUMERIC
fga_status status_reset(Workspace &ws, cudaStream_t s);
fga_status status_check(Workspace &ws, cudaStream_t s, const char *who);
// flag (status word 1) any non-finite value among n reals of type R (precision: FGA_PREC_*)
fga_status flag_nonfinite(Workspace &ws, const void *data, int64_t n, int precision, cudaStream_t s);
// the same for nf fields of nb beams stored with stride cap
fga_status flag_nonfinite_state(Workspace &ws, const void *st, int64_t cap, int64_t nb, int nf, int precision,
                                cudaStream_t s);
fga_status run_lattice(Workspace &ws, const LatticePlan &plan, int precision, const void *rec, double k, double rw,
                       void *u, cudaStream_t s, int cat = P_GATHER, const float *amax = nullptr);
int64_t read_lattice_pair_counter(bool reset);

fga_status sort_keys_to_perm(Workspace &ws, int32_t *keys, int64_t n, int nbuckets, int32_t **perm_out,
                             int32_t *cell_start, cudaStream_t s);
fga_status build_sum_plan(Workspace &ws, const BinGrid &g, const int32_t *cell_start_dev, int nclasses,
                          const double *pts_host, int64_t npts, cudaStream_t s, SumPlan &plan);
fga_status run_sum(Workspace &ws, const SumPlan &plan, int precision, const void *rec_sorted, const double *pts_dev,
                   double k, double rw, void *u_out, cudaStream_t s, int cat = P_GATHER);
// bucket starts copied to the host by build_sum_plan (valid after it returns)
const int32_t *plan_host_cell_start(const Workspace &ws);

// acc += a * b for complex a, b as two fused multiply-add chains (the compiler may not reassociate
// acc + (ar br - ai bi) into FMAs itself)
template <typename R> __device__ __forceinline__ void cmac(R &accr, R &acci, R ar, R ai, R br, R bi) {
    accr = fma(ar, br, accr);
    accr = fma(-ai, bi, accr);
    acci = fma(ar, bi, acci);
    acci = fma(ai, br, acci);
}

// exp(am) * (cos ph, sin ph).  FP32: Cody-Waite reduction of ph by 2 pi (two-part constant), then
// the hardware sine/cosine and exponential approximations; FP64: the libm-accurate functions.
template <typename R> __device__ __forceinline__ void gauss_phase_exp(R ph, R am, R *er, R *ei);
template <> __device__ __forceinline__ void gauss_phase_exp<float>(float ph, float am, float *er, float *ei) {
    constexpr double TWO_PI = 6.283185307179586476925286766559;
    constexpr float TP_HI = (float)TWO_PI;
    constexpr float TP_LO = (float)(TWO_PI - (double)TP_HI);
    constexpr float INV_TP = (float)(1.0 / TWO_PI);
    const float n = rintf(ph * INV_TP);
    float r = fmaf(-n, TP_HI, ph);
    r = fmaf(-n, TP_LO, r);
    float s, c;
    __sincosf(r, &s, &c);
    const float e = __expf(am);
    *er = e * c;
    *ei = e * s;
}
template <> __device__ __forceinline__ void gauss_phase_exp<double>(double ph, double am, double *er, double *ei) {
    double s, c;
    sincos(ph, &s, &c);
    const double e = exp(am);
    *er = e * c;
    *ei = e * s;
}

}  // namespace fga
