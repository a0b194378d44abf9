/*
 * fga.h -- C ABI of the GB300 (sm_103a) frozen Gaussian approximation library.
 *
 * Method: Hateley, Chai, Tong & Yang, "Frozen Gaussian approximation for 3-D elastic wave
 * equation and seismic tomography" (arXiv:1810.06760).  The library computes the method's three
 * data-parallel steps (Fig. fig:FGA_alg) on one GPU:
 *   1. decomposition of the initial displacement f and velocity g into Gaussian packets on a
 *      tensor (q,p) mesh (Eqs. psi, alpha^k);
 *   2. time propagation of every packet ("beam") by classical RK4: rays (Eqs. char_plus,
 *      char_minus), dzQ/dzP (Eq. DzDt), amplitudes with the SV/SH coupling (Eqs. amp_P, amp_SV,
 *      amp_SH);
 *   3. reconstruction by the truncated Gaussian sum of Eq. FGA at points.
 *
 * Conventions
 *  - Every call is asynchronous on the caller's CUDA stream `s` unless it says otherwise; the
 *    caller owns every buffer it passes.  Pointers marked DEVICE must be device memory of the
 *    current device; pointers marked HOST are read before the call returns.
 *  - Complex numbers are interleaved (re, im).  Arrays of 3-vectors are [n][3] row-major.
 *  - Every call returns an fga_status; no C++ exception crosses the ABI.  fga_last_error()
 *    gives a message for the last failing call of the calling thread.
 *  - Precision is chosen per beam set: FGA_PREC_FP32 (ray, amplitude and sum arithmetic in
 *    FP32) or FP64.  Outputs of a beam set are complex64 (FP32) or complex128 (FP64).
 *  - Beam classes: 0 = P "+", 1 = P "-", 2 = S "+", 3 = S "-" (the two-way propagation of
 *    Eqs. char_plus / char_minus).  An S beam carries both SV and SH amplitudes.
 */
#ifndef FGA_H
#define FGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fga_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    FGA_OK = 0,
    FGA_ERR_INVALID_ARG = 1, /* bad size, pointer, descriptor field; nothing was launched */
    FGA_ERR_OOM = 2,         /* a device allocation failed; nothing was launched */
    FGA_ERR_CUDA = 3,        /* a CUDA runtime call failed; the message has the CUDA error */
    FGA_ERR_TIMEOUT = 4,     /* a bounded wait ran out */
    FGA_ERR_NUMERIC = 5,     /* non-finite values in the beam state or the results (fga_solve) */
    FGA_ERR_UNSUPPORTED = 6, /* valid request the library does not implement */
    FGA_ERR_CANCELLED = 7    /* a served request was cancelled (fga_server_cancel) */
} fga_status;

enum { FGA_PREC_FP32 = 0, FGA_PREC_FP64 = 1 };

enum {
    FGA_MEDIUM_CONST = 0,  /* constant c_p, c_s */
    FGA_MEDIUM_SINE = 1,   /* c_p = cp0 + amp sin(2 pi x1) sin(2 pi x2) sin(2 pi x3), c_s = cs_ratio c_p,
                              evaluated exactly with its gradient and Hessian */
    FGA_MEDIUM_GRID = 2,   /* c_p, c_s and their first and second derivatives given on a node
                              grid, trilinearly interpolated (all 10 fields) */
    FGA_MEDIUM_LAYERED = 3 /* piecewise-constant layers between interfaces (Sec. 3.1): parallel planes
                              or concentric spheres (layer_shape) */
};

/* Shape of the interfaces of a layered medium. */
enum { FGA_LAYERS_PLANES = 0, FGA_LAYERS_SPHERES = 1, FGA_LAYERS_UNDULATING = 2 };

/* Velocity model (Eqs. ewe_ps, ps_speed).  Grid media: node (i,j,l) sits at
 * origin + (i*spacing[0], j*spacing[1], l*spacing[2]); positions outside the grid read the nearest
 * boundary value of every field.  Layered media: nlayers <= 8 layers, z_interfaces[nlayers-1]
 * increasing depths (HOST arrays) measured along layer_normal: the interfaces are the planes
 * layer_normal . x = z_interfaces[i].  layer_normal = (0, 0, 0) means (0, 0, 1) (flat layers in x3);
 * any other vector is normalised (tilted layers: the library propagates such a medium in the frame
 * whose third axis is the normal and converts beams, points and results at its boundary).
 * layer_shape = FGA_LAYERS_SPHERES: the interfaces are the spheres |x - layer_center| = z_interfaces[i],
 * radii strictly decreasing and positive (layer 0 lies outside the largest sphere, layer i between
 * spheres i-1 and i; a point on a sphere belongs to the inner side), and layer_normal must be zero.
 * Sec. 3.1 treats an interface of general shape in the local tangent-normal coordinates of the point
 * where a beam meets it, the tangent plane standing in for the flat interface: at each crossing the
 * library rotates the beam into the frame whose third axis is the sphere's normal there, applies the
 * flat-interface conditions (Snell's law, continuity of displacement and traction, the dzQ/dzP jump of
 * Eq. Inter_DzQDzP; the curvature of the sphere does not enter), and rotates the children back.  Beams,
 * points and results stay in global coordinates.
 * layer_shape = FGA_LAYERS_UNDULATING: interface i is the surface
 *   x3 = z_interfaces[i] + layer_amp[i] cos(2 pi x1 / layer_wavelength[0]) cos(2 pi x2 / layer_wavelength[1])
 * (z_interfaces increasing, wavelengths > 0, and neighbouring surfaces apart: |a_i| + |a_i+1| <
 * z_i+1 - z_i, so that the layers are not parallel but never touch).  A point lies in the layer given by the
 * number of surfaces at or above it; a crossing is handled as for spheres, in the frame of the surface's
 * normal at the crossing point.  layer_normal must be zero. */
typedef struct {
    int kind;
    double cp0, cs0;
    double amp, cs_ratio;
    int n[3];
    double origin[3], spacing[3];
    int nlayers;
    const double *z_interfaces, *layer_cp, *layer_cs, *layer_rho;
    double layer_normal[3];
    int layer_shape;
    double layer_center[3];
    double layer_amp[8];
    double layer_wavelength[2];
} fga_model_desc;

typedef struct fga_model fga_model;
typedef struct fga_beams fga_beams;

/* Create a model.  For FGA_MEDIUM_GRID, grid_p and grid_s are DEVICE float arrays of
 * n[0]*n[1]*n[2]*10 values, node-major (axis 0 slowest), fields per node
 * c, dc/dx1, dc/dx2, dc/dx3, c_11, c_12, c_13, c_22, c_23, c_33; they are copied into the
 * library's own layout (the caller may free them after the call's stream work completes).
 * Other kinds take NULL.  Errors: INVALID_ARG (kind, sizes, spacing <= 0, nlayers > 8, interface depths
 * not increasing or radii not decreasing, a bad layer_shape, a layer without c_p > c_s > 0 and rho > 0,
 * undulating surfaces that may touch), OOM. */
fga_status fga_model_create(fga_model **out, const fga_model_desc *desc, const float *grid_p,
                            const float *grid_s, fga_stream_t s);
fga_status fga_model_destroy(fga_model *m);

/* Decomposition input (Eqs. psi, alpha^k).
 *  f, g: DEVICE complex128 arrays [ny0][ny1][ny2][3] sampling the initial displacement and
 *        velocity at y0 + (i dy0, j dy1, l dy2); g may be NULL (zero velocity).
 *  Mesh: q_{d,i} = q0[d] + i dq[d] (nq per axis), p_{d,j} = p0[d] + j dp[d] (np per axis);
 *        mesh index = ((iq0 nq + iq1) nq + iq2) np^3 + (jp0 np + jp1) np + jp2.
 *  class_mask: bit c creates the beams of class c at every mesh point. */
typedef struct {
    double k;
    int ny[3];
    double y0[3], dy[3];
    const void *f, *g;
    int nq;
    double q0[3], dq[3];
    int np;
    double p0[3], dp[3];
    unsigned class_mask;
    int precision;
    /* layered media only (0 selects the default): a beam is dropped at its (max_interfaces+1)-th
     * interface (default 4); children whose amplitude is below child_rel_min of the incident one
     * are not created (default 1e-6); room is reserved for growth x the initial beam count
     * (default 4; children beyond it are dropped and counted). */
    int max_interfaces;
    double child_rel_min;
    double growth;
    /* beam selection (step 1 of Fig. fig:FGA_alg chooses the sets of beams to propagate): with
     * psi_rel_min > 0 only the beams with |psi| > psi_rel_min x max|psi| are created, |psi| the norm
     * of the beam's psi (P: |psi|; S: (|psi_sv|^2 + |psi_sh|^2)^{1/2}) and the maximum taken over every
     * requested class and mesh point; survivors keep mesh order within their class.  0 keeps every
     * beam; values must lie in [0, 1). */
    double psi_rel_min;
} fga_init_desc;

/* Point-force source of the paper's accuracy experiment (Eq. ex_homo): a force F(t) = force s(t) at
 * x0 in a homogeneous medium (rho, c_p, c_s), s(t) = cos(2 pi f (t + T0)) exp(-(t + T0)^2 / sigma^2)
 * (the source-time function printed with Eq. ex_anal). */
typedef struct {
    double x0[3];
    double force[3];
    double rho, cp, cs;
    double f, T0, sigma;
} fga_point_force;

/* The displacement the point force radiates, Eq. ex_anal (Stokes' solution: far-field P and S terms
 * and the near-field term), and its time derivative, at time t on the grid y0 + (i dy0, j dy1, l dy2):
 * the initial data (f, g) of a decomposition that starts the FGA at time t.  The near-field integral
 * int_{r/c_p}^{r/c_s} tau s(t - tau) dtau uses composite 8-point Gauss-Legendre quadrature on panels of
 * at most 1/(8 f) and sigma/4; du/dt uses its integration-by-parts form.  FP64 throughout.
 *  u_out, v_out: DEVICE complex128 [ny0][ny1][ny2][3] (imaginary parts 0), the layout of
 *                fga_init_desc.f and .g; either may be NULL (not both).  A grid point at the source
 *                itself (r <= 1e-12 (1 + |x0|_1)) gets 0.
 * Asynchronous on s.  Errors: INVALID_ARG (NULL, rho <= 0, not 0 < c_s < c_p, sigma <= 0, f < 0,
 * ny < 1, dy <= 0, non-finite values, more than 2^37 points), CUDA. */
fga_status fga_point_force_field(const fga_point_force *src, const int ny[3], const double y0[3], const double dy[3],
                                 double t, void *u_out, void *v_out, fga_stream_t s);

/* Steps 1 of Fig. fig:FGA_alg: the wave-packet transform F(q,p) = sum_y f(y) exp(-i k p.(y-q)
 * - k|y-q|^2/2) dy^3 (and G from g) as three per-axis contractions, then one beam per mesh point
 * and requested class with Q = q, P = p, dzQ = I, dzP = -iI (Z = 2I) and amplitude
 * 2^{3/2} psi, psi = (F.n +- i G.n/(k c(q) |p|))/2 (Eq. alpha^k read with |p|; n = p/|p| for P,
 * the SV and SH directions for S); with psi_rel_min > 0 only the selected beams (see above).
 * Allocates the beam set (freed by fga_beams_destroy); the selection first evaluates psi for
 * every mesh point and class (no beam storage) and then allocates only the survivors.
 * Errors: INVALID_ARG (k <= 0, sizes, empty mask, psi_rel_min outside [0, 1)), OOM, CUDA. */
fga_status fga_decompose(const fga_model *m, const fga_init_desc *init, fga_beams **out, fga_stream_t s);

/* The wave-packet transform of Eq. psi alone (the first half of step 1):
 *   F(q,p) = sum_y f(y) exp(-i k p.(y-q) - k|y-q|^2/2) dy0 dy1 dy2
 * of init->f on init's (q,p) mesh, computed as fga_decompose computes it (three per-axis complex
 * contractions; FP16-split tensor-core products with FP32 accumulation for FGA_PREC_FP32, FP64 for
 * FGA_PREC_FP64).  init->g, class_mask and the layered options are ignored.
 *  F_out: DEVICE complex [A][A][A][3] (A = nq np), complex64 for FP32 and complex128 for FP64, in the
 *         per-axis pair layout: entry (a0, a1, a2) with a_d = iq_d np + jp_d holds F at
 *         q_d = q0[d] + iq_d dq[d], p_d = p0[d] + jp_d dp[d].
 * Uses library-owned temporaries (allocated and released inside the call); synchronises s.
 * Errors: INVALID_ARG (k <= 0, sizes, spacings, NULL pointers), OOM, TIMEOUT (a tensor-core wait ran
 * out), CUDA. */
fga_status fga_transform(const fga_init_desc *init, void *F_out, fga_stream_t s);

/* Step 2: advance every beam nsteps classical RK4 steps of size dt (dt may be negative).
 * Errors: INVALID_ARG (nsteps < 0, dt not finite), CUDA. */
fga_status fga_propagate(const fga_model *m, fga_beams *b, double dt, int nsteps, fga_stream_t s);

/* Step 3 at the current beam state: u(x) = sum over beams with |x - Q| <= rw of
 * w a N exp(i k P.(x-Q) - k|x-Q|^2/2), w = dq^3 dp^3 / (2 pi/k)^{9/2} (Eq. FGA), N the
 * polarisation (P/|P| for P; a_sv N_sv + a_sh N_sh for S).  rw <= 0 selects 6/sqrt(k).
 *  x: DEVICE float64 [n][3];  u_out: DEVICE complex [n][3] (complex64 for FP32 beams, complex128
 *  for FP64).  n = 0 is a no-op.  Uses library-owned scratch memory (allocated on demand).
 *  Errors: INVALID_ARG, OOM, CUDA. */
fga_status fga_reconstruct(const fga_beams *b, const double *x, int64_t n, double rw, void *u_out,
                           fga_stream_t s);

/* A tensor lattice of points x_{ijl} = (axis[0][i], axis[1][j], axis[2][l]) (HOST arrays of n[d]
 * increasing coordinates).  Results on a lattice are stored [i][j][l][3] (l fastest). */
typedef struct {
    int n[3];
    const double *axis[3];
} fga_lattice;

/* Step 3 on a lattice (snapshot grids, receiver arrays): the same sum as fga_reconstruct at the
 * lattice points, evaluated with the per-axis factorisation exp(i k P.(x-Q) - k|x-Q|^2/2) =
 * prod_d exp(i k P_d (x_d-Q_d) - k (x_d-Q_d)^2/2) of Eq. FGA's Gaussian.  u_out: DEVICE complex
 * [n0][n1][n2][3].  Synchronises s (FP32 beams: to read the call's own error word of the tensor-core
 * sum).  Errors: INVALID_ARG (empty axis, non-increasing axis), OOM, TIMEOUT (a bounded wait of the
 * tensor-core sum ran out; u_out is then incomplete), CUDA. */
fga_status fga_reconstruct_lattice(const fga_beams *b, const fga_lattice *lat, double rw, void *u_out,
                                   fga_stream_t s);

/* Step 3 at points given in spherical coordinates (Sec. 3, layered-Earth example: only the x of
 * Eq. FGA changes, every other step is coordinate free): point q = (r, theta, phi), r the distance to
 * the origin (the Earth's centre), theta the longitude and phi the latitude in radians, is summed at
 *   x = (r cos(theta) cos(phi), r sin(theta) cos(phi), r sin(phi)).
 * The conversion runs on the device in FP64; otherwise as fga_reconstruct.
 *  rtp: DEVICE float64 [n][3];  u_out: DEVICE complex [n][3] (Cartesian components of u).
 *  Errors: INVALID_ARG, OOM, CUDA. */
fga_status fga_reconstruct_spherical(const fga_beams *b, const double *rtp, int64_t n, double rw, void *u_out,
                                     fga_stream_t s);

/* The same sum as fga_reconstruct, for callers that may not allocate device memory: code running
 * where cudaMalloc/cudaFree are unavailable or unsafe (a host callback, a real-time loop that must
 * not stall on the allocator's implicit synchronisation, a plug-in handed buffers by an outside
 * memory pool).  The paper has no counterpart; this is a service of the library.
 * It allocates nothing: its only scratch is a fixed 12 MiB device array inside the library (held by
 * every GPU that loads the library until the process exits).  It tests every beam against every
 * point (no binning), so it suits modest beam counts; n must be <= 4096 (larger n is rejected with
 * FGA_ERR_INVALID_ARG and a message).  The first call on each device looks up the scratch array's
 * address; that lookup may load the library's module on the device and place the 12 MiB array (a
 * one-time cost that can synchronise the device), so make the first call -- a call with n = 0 does
 * only this set-up -- before any stream capture or stall-free section.  All calls share the scratch array:
 * calls that overlap on the GPU (e.g. on two streams) race; calls ordered on one stream do not.
 * Nothing in the scratch has to start at zero (each call overwrites what it reads).
 *  x: DEVICE float64 [n][3]; u_out: DEVICE complex [n][3] in the beams' precision. */
fga_status fga_reconstruct_noalloc(const fga_beams *b, const double *x, int64_t n, double rw, void *u_out,
                                   fga_stream_t s);

/* Whole forward solve: decompose, propagate nsteps of dt, and sum at the sample times.
 *  times: HOST, n_times increasing values in (0, nsteps*dt]; a sample inside step n uses cubic
 *         Hermite interpolation of Q and P and linear interpolation of the amplitudes.
 *  rx:    DEVICE float64 [n_rx][3]; seis_out DEVICE complex [n_times][n_rx][3] (may be NULL if
 *         n_rx = 0).  Or rx_lattice (non-NULL): receivers on a lattice, n_rx and rx ignored,
 *         seis_out [n_times][n0][n1][n2][3].
 *  snap:  DEVICE float64 [n_snap][3] summed at t = nsteps*dt into snap_out DEVICE complex
 *         [n_snap][3] (may be NULL if n_snap = 0).  Or snap_lattice (non-NULL): n_snap and snap
 *         ignored, snap_out [n0][n1][n2][3].
 *  rw <= 0 selects 6/sqrt(k).  Device memory: the beam set, its sorted copy and a buffer of
 *  reconstruction records of up to 48 GB (at most 40% of the free memory) per window of steps.
 *  Synchronous: returns after the stream has finished the solve.
 *  Errors: INVALID_ARG, OOM, CUDA, NUMERIC (a non-finite value in the final beam state, the seismograms
 *  or the snapshot; the outputs are then unreliable), TIMEOUT (a bounded wait of the tensor-core
 *  Gaussian sum ran out; the outputs are incomplete). */
typedef struct {
    double dt;
    int nsteps;
    int n_times;
    const double *times;
    int64_t n_rx;
    const double *rx;
    int64_t n_snap;
    const double *snap;
    double rw;
    const fga_lattice *rx_lattice;
    const fga_lattice *snap_lattice;
    /* FGA_COORDS_CARTESIAN (0, the default of a zeroed descriptor) or FGA_COORDS_SPHERICAL: the point
     * arrays rx and snap then hold (r, theta, phi), converted in the library as fga_reconstruct_spherical
     * does (lattices are Cartesian only). */
    int coords;
} fga_solve_desc;

enum { FGA_COORDS_CARTESIAN = 0, FGA_COORDS_SPHERICAL = 1 };

fga_status fga_solve(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd,
                     void *seis_out, void *snap_out, fga_stream_t s);

/* Beam bookkeeping.  fga_beams_count: HOST int64 n_by_class[4] (synchronises the stream the
 * beams were last used on).  fga_beams_export: copies the state to HOST in mesh order, per beam
 * 48 float64 = Q(3), P(3), dzQ (3x3 complex, [m][j] = dQ_j/dz_m), dzP (3x3 complex), amplitudes
 * (3 complex: P: a, 0, 0; S: a_sv, a_sh, 0), and HOST int32 meta per beam (bits 0-1 class, bit 2
 * S frame reference e1); either pointer may be NULL.  Synchronous. */
fga_status fga_beams_count(const fga_beams *b, int64_t *n_by_class);
fga_status fga_beams_export(const fga_beams *b, double *state_host, int32_t *meta_host);
fga_status fga_beams_destroy(fga_beams *b);

/* The parameters a beam set was made with: HOST k, the quadrature weight w = prod_d(dq_d dp_d)/(2 pi/k)^{9/2}
 * of Eq. FGA, and the precision; any pointer may be NULL. */
fga_status fga_beams_params(const fga_beams *b, double *k, double *w, int *precision);

/* A beam set from exported beams (to resume a propagation, or to propagate beams made elsewhere): n beams,
 * HOST state [n][48] float64 in the fga_beams_export layout (the last two values ignored), HOST meta
 * int32 [n] with only the class (bits 0-1) and S-frame (bit 2) bits, and the k, w and precision of the
 * set they came from (fga_beams_params).  Beams are grouped by class, keeping their order within a
 * class; the Q compensation starts at zero.  Smooth media only (a layered population carries lineage
 * and layer bits).  Synchronous.  Errors: INVALID_ARG (counts, k or w <= 0, other meta bits), OOM, CUDA. */
fga_status fga_beams_import(int64_t n, const double *state, const int32_t *meta, double k, double w, int precision,
                            fga_beams **out, fga_stream_t s);

/* All live beams in storage order (the form for layered media, where beams split at interfaces).
 * Writes up to cap beams: HOST state [n][48] (as fga_beams_export), meta int32 [n] (bits 0-1 class,
 * 2 S frame e1, 4-7 layer, 8-11 interfaces crossed, 13-14 class of the initial beam of the lineage),
 * mesh_id int64 [n] (the mesh point the beam descends from; with bits 13-14 of meta it names the
 * initial beam), path int64 [n] (lineage: 0 for an initial beam, parent*4 + child + 1 for a child,
 * child 0 reflected P, 1 reflected S, 2 transmitted P, 3 transmitted S); *n_out = live beams (may
 * exceed cap; nothing beyond cap is written); *dropped = children lost to the reserved capacity.
 * Synchronous. */
fga_status fga_beams_export_all(const fga_beams *b, int64_t cap, int64_t *n_out, int64_t *dropped, double *state,
                                int32_t *meta, int64_t *mesh_id, int64_t *path);

/* Serving loop for forward solves (no counterpart in the paper; the paper runs one solve at a time).
 * Requests (a decomposition descriptor plus a solve descriptor, as for fga_solve, each with its own
 * source data, k, mesh, sample times and receivers) share one resident model.  A request's peak
 * device memory is estimated from its sizes; requests start in submission order while the running
 * ones fit hbm_budget_bytes (<= 0: 85% of the free device memory at creation); one that exceeds the
 * budget on its own runs when nothing else runs.  n_workers threads each own a non-blocking stream
 * and run one request at a time, so up to n_workers solves share the GPU; record_cap_bytes (<= 0:
 * 2e9) caps each solve's per-window record buffer.  The caller keeps every buffer a request names
 * (f, g, receivers, snapshot points, outputs; all DEVICE as for fga_solve) alive and untouched until
 * fga_server_wait returns for it; the times array and lattice descriptors (with their host axes) are copied
 * at submission.  Layered media are not
 * served.  Kernel profiling (fga_profile_enable) must be off while a server runs.
 *  fga_server_wait blocks until the request is done (timeout_s <= 0: no limit; else FGA_ERR_TIMEOUT),
 *  returns the request's own status and fills info (may be NULL); a request id can be waited once.
 *  fga_server_destroy finishes the queued requests, then stops the workers. */
typedef struct {
    int n_workers;
    double hbm_budget_bytes;
    double record_cap_bytes;
    /* admission order: FGA_SERVE_FIFO (0, submission order) or FGA_SERVE_SHORTEST (the queued request
     * with the least estimated work, beams x steps, first; a request queued for longer than
     * age_limit_s (<= 0: 2 s) goes first, oldest first, so that no request starves) */
    int policy;
    double age_limit_s;
} fga_server_desc;

enum { FGA_SERVE_FIFO = 0, FGA_SERVE_SHORTEST = 1 };

typedef struct {
    int status;       /* the request's fga_status */
    int worker;       /* worker that ran it */
    double t_submit;  /* seconds since the server was created (host steady clock) */
    double t_start;
    double t_end;     /* after the request's stream drained */
    double bytes;     /* estimated peak device memory */
    int64_t beams;
} fga_request_info;

typedef struct {
    int64_t queued;
    int64_t running;
    int64_t completed;
    int64_t peak_running;
    double inflight_bytes;
    double peak_bytes;
    double budget_bytes;
} fga_server_stats_t;

typedef struct fga_server fga_server;
fga_status fga_server_create(fga_server **out, const fga_model *m, const fga_server_desc *d);
fga_status fga_server_submit(fga_server *sv, const fga_init_desc *init, const fga_solve_desc *sd, void *seis_out,
                             void *snap_out, int64_t *id);
fga_status fga_server_wait(fga_server *sv, int64_t id, double timeout_s, fga_request_info *info);
fga_status fga_server_stats(fga_server *sv, fga_server_stats_t *out);
/* Cancel a request: a queued one is dropped at once, a running one stops at its next window of steps
 * (its outputs are then incomplete).  Its fga_server_wait returns FGA_ERR_CANCELLED; a request that has
 * already finished keeps its own status.  Errors: INVALID_ARG (unknown or collected id). */
fga_status fga_server_cancel(fga_server *sv, int64_t id);
fga_status fga_server_destroy(fga_server *sv);

/* Reverse mode of fga_solve's seismograms (no counterpart in the paper, which uses the method as the
 * forward model of tomography and waveform inversion and leaves the adjoint to that literature).
 * For a cotangent ubar of the seismograms, DEVICE complex [n_times][n_rx][3] in the init
 * precision (dL/dRe u + i dL/dIm u; ubar = u - d for L = 1/2 sum |u - d|^2), ADDS dL/d(node field)
 * to grad_p and grad_s, DEVICE float64 arrays shaped like the model grids, [n0][n1][n2][10] in the
 * field order of fga_model_create (the caller zeroes them first; several sources may accumulate).
 * L is the discrete forward map fga_solve computes: initialisation (its c(q) term), classical RK4,
 * Hermite-interpolated records and the windowed Gaussian sums (the window's edge is not
 * differentiated).  The forward pass stores the beam state every checkpoint_every steps (<= 0: 20);
 * each segment is recomputed in reverse, so device memory holds (ceil(nsteps/C) + C + 7) beam states
 * (46 values per beam) plus 432 values per beam of reverse-step scratch (stage records of 8 steps).  Grid and constant media (constant media have no node fields: grad_p and
 * grad_s may be NULL); receivers as points (sd->rx, sd->n_rx >= 1); snapshots are ignored; at most
 * 4 sample times inside one step and n_rx * (3 + 6 * samples in a step) values of the init
 * precision within 200 KiB.  Node cotangents of a beam are summed along its path over up to 8 steps
 * per trilinear cell, then accumulated with atomics (FP64 path: FP64 into the outputs; FP32 path:
 * FP32 into a scratch grid that is added to the outputs at the end), so the last bits depend on the
 * order of the updates.  Synchronous on s.  Errors: INVALID_ARG, UNSUPPORTED
 * (other media), OOM, CUDA; INVALID_ARG also for a beam selection (psi_rel_min > 0), whose
 * surviving set is not differentiated. */
fga_status fga_solve_vjp(const fga_model *m, const fga_init_desc *init, const fga_solve_desc *sd, const void *ubar,
                         double *grad_p, double *grad_s, int checkpoint_every, fga_stream_t s);

/* Cross-correlation traveltime misfit and its adjoint source.  The paper's inversion section
 * (wave-equation-based traveltime tomography and FWI) measures traveltimes as in Tromp, Tape and
 * Liu (2005) and prints no formula; this is that measurement on the sampled records.
 * syn, obs: DEVICE complex [n_times][n_rx][3] (the seismogram layout of fga_solve), complex64 for
 * FGA_PREC_FP32 and complex128 for FGA_PREC_FP64, samples dt apart.  Per receiver r, with
 * C_r(m) = sum_j sum_c Re(conj(syn[j][r][c]) obs[j+m][r][c]) for m = -max_lag..max_lag (zero
 * beyond the record) and m* the smallest lag of its largest value:
 *   tau[r] = (m* + (a - c) / (2 (a - 2b + c))) dt   with a, b, c = C_r(m*-1), C_r(m*), C_r(m*+1),
 * the step taken only when -max_lag < m* < max_lag and a - 2b + c < 0 (tau > 0: the observed
 * record arrives later).  misfit = 1/2 sum_r tau[r]^2 (DEVICE double [1], may be NULL).
 * ubar (DEVICE, the type and layout of syn, may be NULL) receives the misfit's cotangent
 * dL/dRe syn + i dL/dIm syn in the synthetic-only form: ubar[j][r][c] = tau[r] s'[j] dt / N_r with
 * s'[j] = (syn[j+1] - syn[j-1]) / (2 dt), N_r = (1/dt) sum_{j=-1}^{n_times-1} sum_c
 * |syn[j+1] - syn[j]|^2 and syn[-1] = syn[n_times] = 0 (0 where N_r = 0).  It is the exact
 * derivative of tau when obs is a whole-sample shift of syn; fed to fga_solve_vjp it gives the
 * traveltime misfit's model gradient.  tau: DEVICE double [n_rx].  The correlation and tau are
 * computed in FP64 for both precisions.  Non-finite records give unspecified delays.  Needs
 * 96 n_times + 16 max_lag + 8 bytes within 200 KiB of shared memory.  Asynchronous on s.
 * Errors: INVALID_ARG (precision, n_times < 1, n_rx < 0, dt, max_lag outside [0, n_times),
 * missing pointers, record too long), CUDA. */
fga_status fga_traveltime_adjoint(const void *syn, const void *obs, int precision, int64_t n_times, int64_t n_rx,
                                  double dt, int max_lag, double *tau, void *ubar, double *misfit, fga_stream_t s);

/* Cell binning (no counterpart in the paper: the fast summation it cites is not printed).
 * For FP32 centres Q (DEVICE float [n][3]) computes key = (c0 nc1 + c1) nc2 + c2 with
 * c_d = floor((Q_d - o_d) * inv_h) in FP32 round-to-nearest, clamped to [0, nc_d-1], then a
 * stable sort: perm (DEVICE int32 [n]) lists the beams cell by cell in increasing index,
 * cell_start (DEVICE int32 [ncells+1]) the cell offsets; keys (DEVICE int32 [n]) may be NULL.
 * Uses library-owned scratch.  Errors: INVALID_ARG (n < 0, nc_d < 1, ncells >= 2^24), OOM, CUDA. */
fga_status fga_bin(const float *Q, int64_t n, const float origin[3], float inv_h, const int nc[3],
                   int32_t *keys, int32_t *perm, int32_t *cell_start, fga_stream_t s);

/* Profiling of the library's own kernels (no counterpart in the paper; used to measure it).
 * mode 0: off (default); 1: launch and work counters, including the in-window pair count (which
 * adds a few instructions to the Gaussian-sum kernels); 2: launch counters plus the device time of
 * every kernel launch, taken with CUDA events recorded on the launching stream around it (no pair
 * count); 3: both.  Categories of
 * count[] / ms[]: 0 decomposition, 1 RK4 propagation, 2 binning (keys, sort, permutation),
 * 3 records, 4 Gaussian sums at sample times inside fga_solve, 5 Gaussian-sum reductions,
 * 6 Gaussian sums at the current beam state (snapshots, fga_reconstruct, fga_reconstruct_lattice),
 * 7 layered-medium steps with interface events, 8 adjoint forward recomputation (checkpoints and
 * segments), 9 adjoint reverse steps, 10 adjoint initial-amplitude term, 11 traveltime misfit.  pairs_in_window counts the
 * (beam, point) pairs inside the truncation window that the Gaussian sum evaluated; pairs_tested the
 * pairs it examined; beam_steps the beam RK4 steps advanced.  fga_profile_read waits for the timed
 * launches to finish; reset != 0 zeroes the counters afterwards.  Process-wide state, meant to be
 * driven from one host thread. */
typedef struct {
    int64_t launches;
    int64_t count[12];
    double ms[12];
    int64_t beam_steps;
    int64_t pairs_in_window;
    int64_t pairs_tested;
} fga_profile_t;
fga_status fga_profile_enable(int mode);
fga_status fga_profile_read(fga_profile_t *out, int reset);

/* Upper bound on the device memory the library allocates for its own buffers (beam sets, sort and
 * record scratch, cached blocks of the serving loop; not the caller's buffers, not the static scratch of
 * fga_reconstruct_noalloc): an allocation that would pass it fails with FGA_ERR_OOM before cudaMalloc
 * is called.  bytes <= 0 removes the bound (the default).  fga_device_memory_in_use reports the bytes
 * currently allocated for such buffers.  Process-wide; meant for hosts that share a GPU, and for testing
 * the out-of-memory paths without exhausting the device. */
fga_status fga_set_device_memory_limit(double bytes);
double fga_device_memory_in_use(void);

/* Message of the last failing call on this thread (always NUL-terminated; truncated to cap). */
void fga_last_error(char *buf, size_t cap);
int fga_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FGA_H */
