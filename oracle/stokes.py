"""FP64 oracle of the analytic wavefield of a point force in a homogeneous elastic medium.

THIS MODULE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It shares no code
with the CUDA library (``paper_1810_06760_gb300``) and never imports it.

The paper's accuracy experiment (Sec. "Accuracy and Parallelizability", Eq. ex_homo) drives
rho u_tt = (lambda + mu) grad div u + mu Laplacian u + F(t) delta(x - x0) and compares with the
analytic solution Eq. ex_anal (Stokes' solution).  With gamma = (x - x0)/r, r = |x - x0|:

  u_i = gamma_i gamma_j F_j(t - r/c_p) / (4 pi rho c_p^2 r)
      + (delta_ij - gamma_i gamma_j) F_j(t - r/c_s) / (4 pi rho c_s^2 r)
      + (3 gamma_i gamma_j - delta_ij) / (4 pi rho r^3)  int_{r/c_p}^{r/c_s} tau F_j(t - tau) dtau,

and the source-time function printed beside it, F_j(t) = d_j s(t) with
s(t) = cos(2 pi f (t + T0)) exp(-(t + T0)^2 / sigma^2) (the paper's F has d = (1, 1, 1)).

The near-field integral is written in closed form, not by quadrature.  With omega = 2 pi f,
g(w) = exp(-w^2/sigma^2 + i omega w) and c0 = t + T0, s(t - tau) = Re g(c0 - tau), and completing
the square, mu = i omega sigma^2 / 2,
  int g dw   = e^{-omega^2 sigma^2 / 4} (sigma sqrt(pi) / 2) erf((w - mu) / sigma)  =: G(w),
  int w g dw = -(sigma^2 / 2) g(w) + mu G(w),
so int_a^b tau s(t - tau) dtau = Re[ c0 (G(w2) - G(w1)) - (int w g)(w2) + (int w g)(w1) ] with
w1 = c0 - b, w2 = c0 - a; the complex error function is scipy's.  The time derivative
du/dt replaces s by s' and the integral by its t-derivative, which integration by parts turns into
a s(t - a) - b s(t - b) + int_a^b s(t - tau) dtau.

Parity status: pinned by ``tests/test_oracle_stokes.py``: the integrals against adaptive quadrature,
the elastic wave equation satisfied by finite differences away from the source, Kelvin's static
solution in the limit of a constant force, the symmetry of the Green's tensor and du/dt against
a finite difference in time.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import erf


@dataclasses.dataclass
class PointForce:
    """A point force d s(t) at x0 in a homogeneous medium (rho, c_p, c_s); s as printed with the
    paper's Eq. ex_anal: cos(2 pi f (t + T0)) exp(-(t + T0)^2 / sigma^2)."""
    x0: np.ndarray
    d: np.ndarray
    rho: float
    cp: float
    cs: float
    f: float
    T0: float
    sigma: float

    # ---- source-time function -----------------------------------------------------------------
    def s(self, t):
        a = np.asarray(t, dtype=np.float64) + self.T0
        return np.cos(2 * math.pi * self.f * a) * np.exp(-(a / self.sigma) ** 2)

    def ds(self, t):
        a = np.asarray(t, dtype=np.float64) + self.T0
        om = 2 * math.pi * self.f
        e = np.exp(-(a / self.sigma) ** 2)
        return (-om * np.sin(om * a) - 2 * a / self.sigma ** 2 * np.cos(om * a)) * e

    # ---- closed-form integrals ----------------------------------------------------------------
    def _g(self, w):
        om = 2 * math.pi * self.f
        return np.exp(-(w / self.sigma) ** 2 + 1j * om * w)

    def _G(self, w):
        om = 2 * math.pi * self.f
        mu = 0.5j * om * self.sigma ** 2
        return (math.exp(-0.25 * (om * self.sigma) ** 2) * 0.5 * self.sigma * math.sqrt(math.pi)
                * erf((w - mu) / self.sigma))

    def near_integral(self, t, a, b):
        """int_a^b tau s(t - tau) dtau (closed form)."""
        om = 2 * math.pi * self.f
        mu = 0.5j * om * self.sigma ** 2
        c0 = np.asarray(t, dtype=np.float64) + self.T0
        w1, w2 = c0 - b, c0 - a
        Ig = self._G(w2) - self._G(w1)
        Iwg = -0.5 * self.sigma ** 2 * (self._g(w2) - self._g(w1)) + mu * Ig
        return np.real(c0 * Ig - Iwg)

    def near_integral_dt(self, t, a, b):
        """d/dt int_a^b tau s(t - tau) dtau = a s(t - a) - b s(t - b) + int_a^b s(t - tau) dtau."""
        c0 = np.asarray(t, dtype=np.float64) + self.T0
        Ig = self._G(c0 - a) - self._G(c0 - b)
        return a * self.s(t - a) - b * self.s(t - b) + np.real(Ig)

    # ---- the wavefield --------------------------------------------------------------------------
    def _field(self, x, t, deriv: bool):
        x = np.atleast_2d(np.asarray(x, dtype=np.float64))
        X = x - np.asarray(self.x0, dtype=np.float64)
        r = np.sqrt(np.sum(X * X, axis=1))
        rs = np.where(r > 0, r, 1.0)
        gam = X / rs[:, None]
        d = np.asarray(self.d, dtype=np.float64)
        gd = gam @ d                                    # gamma_j d_j
        src = self.ds if deriv else self.s
        near = self.near_integral_dt if deriv else self.near_integral
        a, b = r / self.cp, r / self.cs
        fp = src(t - a) / (4 * math.pi * self.rho * self.cp ** 2 * rs)
        fs = src(t - b) / (4 * math.pi * self.rho * self.cs ** 2 * rs)
        fn = near(t, a, b) / (4 * math.pi * self.rho * rs ** 3)
        u = (gam * (gd * fp)[:, None] + (d[None, :] - gam * gd[:, None]) * fs[:, None]
             + (3 * gam * gd[:, None] - d[None, :]) * fn[:, None])
        u[r == 0] = 0.0
        return u

    def displacement(self, x, t):
        """u(x, t) of Eq. ex_anal at points x [n, 3]: real [n, 3]; 0 at the source point."""
        return self._field(x, t, False)

    def velocity(self, x, t):
        """du/dt (x, t): real [n, 3]; 0 at the source point."""
        return self._field(x, t, True)


def e1_source(d=(1.0, 1.0, 1.0), f: float = 1.4702) -> PointForce:
    """The paper's accuracy experiment: x0 = (64, 64, 64) km in a 128 km cube, c_p = 8 km/s,
    c_s = 4.619 km/s, rho = 1, T0 = 0.1768 s, sigma = 0.8660 s, f = 1.4702 Hz."""
    return PointForce(np.array([64.0, 64.0, 64.0]), np.asarray(d, dtype=np.float64), 1.0, 8.0, 4.619, f,
                      0.1768, 0.8660)
