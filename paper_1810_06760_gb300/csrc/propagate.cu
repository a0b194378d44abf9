// A3-A4: per-beam classical RK4 of the FGA ODEs, one thread per beam, the whole state in
// registers for all steps of a launch; reconstruction records written at sample times inside the
// launch's steps.
#include "fga_beam.cuh"

namespace fga {

// out = x + h k over the NF state reals (FP32: pairs as packed FP32x2 FMAs)
template <typename R> __device__ __forceinline__ void axpy_state(R *out, const R *x, R h, const R *kv) {
    if constexpr (sizeof(R) == 4) {
        const float2 h2 = make_float2(h, h);
#pragma unroll
        for (int f = 0; f < NF; f += 2) {
            const float2 r = __ffma2_rn(h2, make_float2(kv[f], kv[f + 1]), make_float2(x[f], x[f + 1]));
            out[f] = r.x;
            out[f + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int f = 0; f < NF; f++) out[f] = x[f] + h * kv[f];
    }
}

// One RHS evaluation per iteration of a single loop, so that the large right-hand side is compiled once
// (four inlined copies overflowed the instruction cache).  Classical RK4 with k1 = f(y_n):
//   e = 0: k2 = f(y + h/2 k1)   acc += h/3 k2,  tmp = y + h/2 k2
//   e = 1: k3 = f(tmp)          acc += h/3 k3,  tmp = y + h k3
//   e = 2: k4 = f(tmp)          acc += h/6 k4 (= y_{n+1}),  tmp = acc
//   e = 3: k1' = f(y_{n+1})     records of the step; y = acc, acc = y + h/6 k1', tmp = y + h/2 k1'
// Iteration -1 is an e = 3 without records: it forms k1 of the first step from y_0.
// The three Q entries of acc hold the step's increment instead (small numbers, rounded at their own
// scale); y_{n+1}'s Q is y_n's plus that increment by compensated summation (kahan_add).
template <typename R, int WAVE, int MED>
__global__ void __launch_bounds__(128) rk4_kernel(ModelDev M, R *__restrict__ st, const int32_t *__restrict__ flags,
                                                  int64_t cap, int64_t beg, int64_t n, R sg, R dt, int nsteps,
                                                  int n_samp, const int *__restrict__ samp_step,
                                                  const R *__restrict__ samp_theta, R w, R *__restrict__ rec,
                                                  int64_t rec_lim, int64_t rec_stride, unsigned *__restrict__ amax) {
    const int64_t b = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= beg + n) return;
    R y[NF], acc[NF], tmp[NF], kk[NF], qc[3];
#pragma unroll
    for (int f = 0; f < NF; f++) {
        y[f] = st[(int64_t)f * cap + b];
        acc[f] = y[f];
        tmp[f] = y[f];
    }
#pragma unroll
    for (int d = 0; d < 3; d++) qc[d] = st[(int64_t)(F_QC + d) * cap + b];
    const bool ref_e1 = (flags[b] & FL_REF_E1) != 0;
    R s0[6];   // Q', P' at y_n (left slopes of the Hermite records)
    int js = 0;
    const R h2 = R(0.5) * dt, h3 = dt / R(3), h6 = dt / R(6);
    for (int it = -1; it < 4 * nsteps; it++) {
        const int e = it & 3;
        beam_rhs<R, WAVE, MED>(M, sg, ref_e1, tmp, kk);
        if (e == 3) {
            if (it >= 0) {
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    R q = y[F_Q + d];
                    kahan_add<R>(q, qc[d], acc[F_Q + d]);
                    acc[F_Q + d] = q;       // acc = y_{n+1} in full
                }
            }
            const int step = it >> 2;
            while (it >= 0 && js < n_samp && samp_step[js] == step) {
                float mloc = 0.f;   // largest |A entry| of this thread's record
                if (b - beg < rec_lim) {
                    R r[REC];
                    beam_record6<R, WAVE>(ref_e1, y, s0, acc, kk, dt, samp_theta[js], w, r);
                    R *dst = rec + ((int64_t)js * rec_stride + (b - beg)) * REC;
#pragma unroll
                    for (int q = 0; q < REC; q++) dst[q] = r[q];
#pragma unroll
                    for (int q = 6; q < REC; q++) mloc = fmaxf(mloc, fabsf((float)r[q]));
                }
                if (amax) {
                    // the sample's bound: maximum over the converged lanes, one atomic by the lowest of them
                    // (non-negative floats order like their bit patterns; a NaN is left to the solve's check)
                    const unsigned mask = __activemask();
                    const unsigned v = __reduce_max_sync(mask, mloc == mloc ? __float_as_uint(mloc) : 0u);
                    if ((int)(threadIdx.x & 31) == __ffs(mask) - 1 && v) atomicMax(amax + js, v);
                }
                js++;
            }
#pragma unroll
            for (int f = 0; f < 6; f++) s0[f] = kk[f];
#pragma unroll
            for (int f = 0; f < NF; f++) y[f] = acc[f];
        }
        // acc += ca kk;  tmp = base + ct kk, base = y (e = 0, 1) or acc before its update (e = 2, 3; y for e = 3)
        const R ca = e < 2 ? h3 : h6;
        const R ct = e == 0 ? h2 : (e == 1 ? dt : (e == 2 ? h6 : h2));
        if (e < 2) {
            axpy_state<R>(tmp, y, ct, kk);
            axpy_state<R>(acc, acc, ca, kk);
        } else if (e == 2) {
            // tmp = y_{n+1} = y + (increment + h/6 k4) on Q
            axpy_state<R>(tmp, acc, ct, kk);
            axpy_state<R>(acc, acc, ca, kk);
#pragma unroll
            for (int d = 0; d < 3; d++) tmp[F_Q + d] = y[F_Q + d] + acc[F_Q + d];
        } else {
            axpy_state<R>(tmp, acc, ct, kk);
            axpy_state<R>(acc, acc, ca, kk);
#pragma unroll
            for (int d = 0; d < 3; d++) acc[F_Q + d] = ca * kk[F_Q + d];   // the new step's increment so far
        }
    }
#pragma unroll
    for (int f = 0; f < NF; f++) st[(int64_t)f * cap + b] = y[f];
#pragma unroll
    for (int d = 0; d < 3; d++) st[(int64_t)(F_QC + d) * cap + b] = qc[d];
}

// records of the current state (theta = 0), gathered in the order of perm (or identity)
template <typename R, int WAVE>
__global__ void records_kernel(const R *__restrict__ st, const int32_t *__restrict__ flags, int64_t cap,
                               const int32_t *__restrict__ perm, int64_t beg, int64_t n, R w, R *__restrict__ rec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = perm ? perm[beg + i] : beg + i;
    R y[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) y[f] = st[(int64_t)f * cap + b];
#pragma unroll
    for (int d = 0; d < 3; d++) y[F_Q + d] -= st[(int64_t)(F_QC + d) * cap + b];   // compensated Q
    R r[REC];
    beam_record<R, WAVE>((flags[b] & FL_REF_E1) != 0, y, y, y, y, R(0), R(0), w, r);
    R *dst = rec + i * REC;
#pragma unroll
    for (int q = 0; q < REC; q++) dst[q] = r[q];
}

template <typename R, int WAVE, int MED>
static void launch_one(const fga_model *m, fga_beams *b, int cls, R dt, int nsteps, const SampleWindow *sw,
                       cudaStream_t s) {
    const int64_t n = b->n_cls[cls];
    if (n == 0) return;
    const int T = 128;
    const int64_t blocks = (n + T - 1) / T;
    const R sg = (cls & 1) ? R(-1) : R(1);
    R *rec = sw ? static_cast<R *>(sw->rec) + sw->rec_off[cls] * REC : nullptr;
    prof_add_beam_steps(n * (int64_t)nsteps);
    ProfScope ps(P_PROP, s);
    rk4_kernel<R, WAVE, MED><<<(unsigned)blocks, T, 0, s>>>(
        m->dev, b->state.as<R>(), b->flags.as<int32_t>(), b->cap, b->off_cls[cls], n, sg, dt, nsteps,
        sw ? sw->n : 0, sw ? sw->step : nullptr, sw ? static_cast<const R *>(sw->theta) : nullptr, (R)b->w, rec,
        sw ? sw->n_in[cls] : 0, sw ? sw->n_rec : 0, (sw && sizeof(R) == 4) ? sw->amax : nullptr);
}

template <typename R, int MED>
static void launch_med(const fga_model *m, fga_beams *b, R dt, int nsteps, const SampleWindow *sw, cudaStream_t s) {
    for (int cls = 0; cls < 4; cls++) {
        if (cls < 2)
            launch_one<R, 0, MED>(m, b, cls, dt, nsteps, sw, s);
        else
            launch_one<R, 1, MED>(m, b, cls, dt, nsteps, sw, s);
    }
}

template <typename R>
static void launch_prec(const fga_model *m, fga_beams *b, R dt, int nsteps, const SampleWindow *sw, cudaStream_t s) {
    switch (m->dev.kind) {
    case FGA_MEDIUM_CONST: launch_med<R, FGA_MEDIUM_CONST>(m, b, dt, nsteps, sw, s); break;
    case FGA_MEDIUM_SINE: launch_med<R, FGA_MEDIUM_SINE>(m, b, dt, nsteps, sw, s); break;
    case FGA_MEDIUM_GRID: launch_med<R, FGA_MEDIUM_GRID>(m, b, dt, nsteps, sw, s); break;
    default: launch_med<R, FGA_MEDIUM_LAYERED>(m, b, dt, nsteps, sw, s); break;
    }
}

fga_status launch_propagate(const fga_model *m, fga_beams *b, double dt, int nsteps, const SampleWindow *sw,
                            cudaStream_t s) {
    if (nsteps <= 0 && (!sw || sw->n == 0)) return FGA_OK;
    if (b->precision == FGA_PREC_FP64)
        launch_prec<double>(m, b, dt, nsteps, sw, s);
    else
        launch_prec<float>(m, b, (float)dt, nsteps, sw, s);
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

fga_status launch_records_from_state(const fga_beams *b, const int32_t *perm, const int64_t beg[4],
                                     const int64_t n_in[4], const int64_t rec_off[4], void *rec, cudaStream_t s) {
    const int T = 256;
    for (int cls = 0; cls < 4; cls++) {
        const int64_t nc = n_in[cls];
        if (nc == 0) continue;
        const unsigned blocks = (unsigned)((nc + T - 1) / T);
        ProfScope ps(P_REC, s);
        if (b->precision == FGA_PREC_FP64) {
            double *dst = (double *)rec + rec_off[cls] * REC;
            if (cls < 2)
                records_kernel<double, 0><<<blocks, T, 0, s>>>(b->state.as<double>(), b->flags.as<int32_t>(), b->cap,
                                                               perm, beg[cls], nc, b->w, dst);
            else
                records_kernel<double, 1><<<blocks, T, 0, s>>>(b->state.as<double>(), b->flags.as<int32_t>(), b->cap,
                                                               perm, beg[cls], nc, b->w, dst);
        } else {
            float *dst = (float *)rec + rec_off[cls] * REC;
            if (cls < 2)
                records_kernel<float, 0><<<blocks, T, 0, s>>>(b->state.as<float>(), b->flags.as<int32_t>(), b->cap,
                                                              perm, beg[cls], nc, (float)b->w, dst);
            else
                records_kernel<float, 1><<<blocks, T, 0, s>>>(b->state.as<float>(), b->flags.as<int32_t>(), b->cap,
                                                              perm, beg[cls], nc, (float)b->w, dst);
        }
    }
    FGA_CUDA(cudaGetLastError());
    return FGA_OK;
}

}  // namespace fga
