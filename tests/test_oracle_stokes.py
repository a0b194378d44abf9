"""Pins of the point-force oracle (Eq. ex_anal, the analytic solution of Eq. ex_homo) against what
the mathematics fixes, independent of the oracle's closed-form integrals:

- the near-field integral and its time derivative against adaptive Gauss-Kronrod quadrature;
- the displacement satisfies the elastic wave equation rho u_tt = (lambda + mu) grad div u + mu Lap u
  away from the source (fourth-order finite differences in space and time), and a 10% error in the
  near-field term, or c_p and c_s exchanged in one term, breaks it by orders of magnitude;
- a force held constant for all time gives Kelvin's static solution
  u_i = d_j [(lambda + 3 mu) delta_ij + (lambda + mu) gamma_i gamma_j] / (8 pi mu (lambda + 2 mu) r);
- the Green's tensor is symmetric (u_i of a force along e_j equals u_j of a force along e_i);
- du/dt equals a finite difference of u in time.
"""
import math

import numpy as np
import pytest

from oracle.stokes import PointForce, e1_source

quad = pytest.importorskip("scipy.integrate").quad


def _args(S):
    return {k: getattr(S, k) for k in ("x0", "d", "rho", "cp", "cs", "f", "T0", "sigma")}


@pytest.mark.parametrize("t,a,b", [(5.0, 1.0, 2.2), (4.0, 0.3, 0.52), (7.0, 3.1, 5.4), (6.93, 4.0, 6.9)])
def test_near_integral_against_quadrature(t, a, b):
    S = e1_source(d=(0.3, -0.5, 0.8))
    q = quad(lambda tau: tau * S.s(t - tau), a, b, epsabs=0, epsrel=1e-12, limit=400)[0]
    qd = quad(lambda tau: tau * S.ds(t - tau), a, b, epsabs=0, epsrel=1e-12, limit=400)[0]
    scale = quad(lambda tau: abs(tau * S.s(t - tau)), a, b, limit=400)[0]
    scale_d = quad(lambda tau: abs(tau * S.ds(t - tau)), a, b, limit=400)[0]
    assert abs(S.near_integral(t, a, b) - q) <= 1e-11 * scale
    assert abs(S.near_integral_dt(t, a, b) - qd) <= 1e-11 * scale_d


def _wave_equation_residual(S, x, t, h=0.02, ht=0.002):
    """max |rho u_tt - (lambda + mu) grad div u - mu Lap u| / max |rho u_tt| by fourth-order stencils."""
    st2 = np.array([-1, 16, -30, 16, -1]) / 12.0
    st1 = np.array([1, -8, 0, 8, -1]) / 12.0
    off = np.arange(-2, 3)
    U = S.displacement
    n = x.shape[0]
    utt = sum(c * U(x, t + o * ht) for c, o in zip(st2, off)) / ht ** 2
    H = np.zeros((n, 3, 3, 3))           # H[:, a, b, i] = d_a d_b u_i
    E = np.eye(3)
    for a in range(3):
        H[:, a, a, :] = sum(c * U(x + o * h * E[a], t) for c, o in zip(st2, off)) / h ** 2
        for b in range(a + 1, 3):
            acc = 0.0
            for ca, oa in zip(st1, off):
                for cb, ob in zip(st1, off):
                    if ca and cb:
                        acc = acc + ca * cb * U(x + oa * h * E[a] + ob * h * E[b], t)
            H[:, a, b, :] = H[:, b, a, :] = acc / h ** 2
    lap = sum(H[:, a, a, :] for a in range(3))
    graddiv = np.stack([sum(H[:, i, j, j] for j in range(3)) for i in range(3)], -1)
    mu = S.rho * S.cs ** 2
    lam = S.rho * S.cp ** 2 - 2 * mu
    R = S.rho * utt - (lam + mu) * graddiv - mu * lap
    return float(np.abs(R).max() / np.abs(S.rho * utt).max())


def _points(S, n=12, seed=1, rmin=8.0, rmax=35.0):
    rng = np.random.default_rng(seed)
    dirs = rng.standard_normal((n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    return S.x0 + dirs * rng.uniform(rmin, rmax, n)[:, None]


@pytest.mark.parametrize("t", [4.0, 5.0, 6.93])
def test_satisfies_elastic_wave_equation(t):
    S = e1_source(d=(0.3, -0.5, 0.8))
    assert _wave_equation_residual(S, _points(S), t) < 1e-6


def test_wave_equation_residual_detects_wrong_terms():
    """The residual pin is sharp: a 10% error in the near-field term, or the S term carrying c_p's
    geometric factor, leaves residuals far above the bar."""
    S = e1_source(d=(0.3, -0.5, 0.8))

    class NearOff(PointForce):
        def near_integral(self, t, a, b):
            return 1.1 * super().near_integral(t, a, b)

    class SwapSpeed(PointForce):
        def displacement(self, x, t):
            u = super().displacement(x, t)
            X = np.atleast_2d(x) - self.x0
            r = np.linalg.norm(X, axis=1)
            gam = X / r[:, None]
            d = np.asarray(self.d)
            perp = d[None, :] - gam * (gam @ d)[:, None]
            fs = self.s(t - r / self.cs)[:, None] / (4 * math.pi * self.rho * r[:, None])
            return u - perp * fs / self.cs ** 2 + perp * fs / self.cp ** 2

    x = _points(S)
    assert _wave_equation_residual(NearOff(**_args(S)), x, 5.0) > 1e-3
    assert _wave_equation_residual(SwapSpeed(**_args(S)), x, 5.0) > 1e-2


def test_constant_force_gives_kelvin_solution():
    """s(t) = exp(-t^2/sigma^2) with f = 0, T0 = 0 and sigma = 1000 s is constant to 1e-5 over the
    times that reach the points, so the field is Kelvin's static solution to that accuracy."""
    S = PointForce(np.array([1.0, 2.0, 3.0]), np.array([0.3, -0.5, 0.8]), 2.5, 6.0, 3.5, 0.0, 0.0, 1000.0)
    x = _points(S, n=20, seed=4, rmin=2.0, rmax=12.0)
    u = S.displacement(x, 3.0)
    mu = S.rho * S.cs ** 2
    lam = S.rho * S.cp ** 2 - 2 * mu
    X = x - S.x0
    r = np.linalg.norm(X, axis=1)
    gam = X / r[:, None]
    want = ((lam + 3 * mu) * S.d[None, :] + (lam + mu) * gam * (gam @ S.d)[:, None]) / (
        8 * math.pi * mu * (lam + 2 * mu) * r[:, None])
    np.testing.assert_allclose(u, want, rtol=1e-4, atol=0)


def test_green_tensor_is_symmetric():
    S = e1_source()
    x = _points(S, n=15, seed=7)
    G = np.stack([PointForce(**{**_args(S), "d": np.eye(3)[j]}).displacement(x, 5.5) for j in range(3)], -1)
    np.testing.assert_allclose(G, np.swapaxes(G, 1, 2), rtol=0, atol=1e-14 * np.abs(G).max())


def test_velocity_is_time_derivative():
    S = e1_source(d=(0.3, -0.5, 0.8))
    x = _points(S, n=15, seed=9)
    ht = 1e-3
    st1 = np.array([1, -8, 0, 8, -1]) / 12.0
    fd = sum(c * S.displacement(x, 5.0 + o * ht) for c, o in zip(st1, range(-2, 3))) / ht
    v = S.velocity(x, 5.0)
    np.testing.assert_allclose(v, fd, rtol=0, atol=1e-8 * np.abs(v).max())
