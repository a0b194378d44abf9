"""FP64 oracle of the cross-correlation traveltime misfit and its adjoint source.

THIS MODULE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It shares no code
with the CUDA library (``paper_1810_06760_gb300``) and never imports it.

The paper's inversion section (Sec. "Wave-equation-based traveltime tomography and FWI") applies
FGA to wave-equation traveltime tomography after Tromp, Tape and Liu (2005).  The delay of the
observed seismogram relative to the synthetic is measured by cross-correlation, the misfit is
half the sum of squared delays, and the adjoint source uses the synthetic alone: a change ds of the
synthetic changes the delay by  int Re(conj(ds/dt) ds) dt / int |ds/dt|^2 dt.  This module writes
those definitions out on the sampled seismograms, in the discretisation the library uses:

  seismograms s (synthetic), d (observed): complex [n_t][n_rx][3], uniform sample spacing dt;
  per receiver r, for lags m = -M..M (zero beyond the record):
      C_r(m) = sum_j sum_c Re( conj(s[j,r,c]) d[j+m,r,c] )
  m* = the smallest lag where C_r is largest;
  for -M < m* < M, with a, b, c = C_r(m*-1), C_r(m*), C_r(m*+1) and den = a - 2b + c:
      delta = (a - c) / (2 den) if den < 0, else 0;   otherwise delta = 0;
  tau_r = (m* + delta) dt                     (tau > 0: the data arrive later than the synthetic);
  s'[j] = (s[j+1] - s[j-1]) / (2 dt)          with s[-1] = s[n_t] = 0 (the zero padding of C);
  N_r   = (1/dt) sum_{j=-1}^{n_t-1} sum_c |s[j+1,r,c] - s[j,r,c]|^2;
  misfit = 1/2 sum_r tau_r^2;
  ubar[j,r,c] = tau_r s'[j,r,c] dt / N_r      (0 where N_r = 0),
the misfit's cotangent in the seismogram convention dL/dRe s + i dL/dIm s.  With these two
difference operators the adjoint source is exactly the derivative of the measured delay when the
data are a whole-sample shift of the synthetic (the parabolic step's numerator holds central
differences of s, its denominator forward differences), which the pins check.

Parity status: pinned by ``tests/test_oracle_traveltime.py`` (exact whole-sample shifts,
antisymmetry under exchanging s and d, zero misfit for identical records, sub-sample shifts of a
smooth pulse, and central finite differences of the measured delay against the adjoint source).
"""
from __future__ import annotations

import numpy as np


def correlation(s, d, max_lag):
    """C[r, m + M] for m = -M..M (FP64), summed over samples and components."""
    s = np.asarray(s, dtype=np.complex128)
    d = np.asarray(d, dtype=np.complex128)
    n_t, n_rx, _ = s.shape
    M = int(max_lag)
    C = np.zeros((n_rx, 2 * M + 1))
    for m in range(-M, M + 1):
        j0, j1 = max(0, -m), min(n_t, n_t - m)
        if j1 <= j0:
            continue
        C[:, m + M] = np.real(np.conj(s[j0:j1]) * d[j0 + m:j1 + m]).sum(axis=(0, 2))
    return C


def delays(s, d, dt, max_lag):
    """tau [n_rx]: the cross-correlation delay of d relative to s, parabolic sub-sample step."""
    C = correlation(s, d, max_lag)
    M = int(max_lag)
    tau = np.zeros(C.shape[0])
    for r in range(C.shape[0]):
        k = int(np.argmax(C[r]))          # first maximum: the smallest lag
        m = k - M
        delta = 0.0
        if -M < m < M:
            a, b, c = C[r, k - 1], C[r, k], C[r, k + 1]
            den = a - 2.0 * b + c
            if den < 0.0:
                delta = (a - c) / (2.0 * den)
        tau[r] = (m + delta) * dt
    return tau


def slope(s, dt):
    """Central differences in time with zero padding at both ends."""
    s = np.asarray(s, dtype=np.complex128)
    p = np.zeros((s.shape[0] + 2,) + s.shape[1:], dtype=np.complex128)
    p[1:-1] = s
    return (p[2:] - p[:-2]) / (2.0 * dt)


def norm_n(s, dt):
    """N [n_rx] = (1/dt) sum over the padded forward differences of |s[j+1] - s[j]|^2."""
    s = np.asarray(s, dtype=np.complex128)
    p = np.zeros((s.shape[0] + 2,) + s.shape[1:], dtype=np.complex128)
    p[1:-1] = s
    return (np.abs(p[1:] - p[:-1]) ** 2).sum(axis=(0, 2)) / dt


def traveltime_adjoint(s, d, dt, max_lag):
    """(tau [n_rx], ubar [n_t][n_rx][3] complex, misfit) for the misfit 1/2 sum tau^2."""
    tau = delays(s, d, dt, max_lag)
    sd = slope(s, dt)
    N = norm_n(s, dt)
    g = np.where(N > 0.0, tau * dt / np.where(N > 0.0, N, 1.0), 0.0)
    ubar = sd * g[None, :, None]
    return tau, ubar, 0.5 * float(np.sum(tau * tau))
