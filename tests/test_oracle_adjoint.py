"""Pins of the oracle's reverse mode (the paper prints no adjoint; the discrete one is checked by
central finite differences of the discrete forward map, in FP64).

* dy/dt: state cotangent against a directional difference, node-field cotangents against
  single-entry differences (dy/dt is linear in the fields, so those agree to rounding);
* the whole solve (initialisation with a velocity term, RK4, Hermite-interpolated records at
  interior and step-end samples, windowed Gaussian sums): gradient of the L2 misfit
  L = 1/2 sum |u - d|^2 with respect to single grid entries and along random directions.
Sources sit off the grid's planes: trilinear interpolation is not differentiable across cell faces,
so a beam held on a face by symmetry has one-sided derivatives only."""
import math

import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import oracle_mesh


def _grid(n=9):
    gp = W.sine_fields_on_nodes(n, 2.0, 0.2)
    gs = (gp.astype(np.float64) / math.sqrt(3.0)).astype(np.float32)
    return gp, gs, 1.0 / (n - 1)


def _rand_state(rng, cls):
    y = np.zeros(48)
    y[0:3] = rng.uniform(0.2, 0.8, 3)
    y[3:6] = rng.normal(size=3) * 3
    DQ = np.eye(3) + 0.2 * (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
    DP = -1j * np.eye(3) + 0.2 * (rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3)))
    y[6:24] = np.stack([DQ.real, DQ.imag], -1).reshape(-1)
    y[24:42] = np.stack([DP.real, DP.imag], -1).reshape(-1)
    a = rng.normal(size=3) + 1j * rng.normal(size=3)
    a[1 if cls < 2 else 2:] = 0
    y[42:48] = np.stack([a.real, a.imag], -1).reshape(-1)
    return y


@pytest.mark.parametrize("mt", [0, 1, 2, 3, 2 | 4, 3 | 4])
def test_rhs_vjp_matches_differences(oracle, mt):
    O = oracle
    gp, gs, h = _grid()
    m = O.Model("grid", grid_p=gp, grid_s=gs, spacing=(h, h, h))
    rng = np.random.default_rng(10 + mt)
    cls = mt & 3
    y = _rand_state(rng, cls)
    live = 42 + (2 if cls < 2 else 4)
    fb = rng.normal(size=48)
    fb[live:] = 0
    yb, gpb, gsb = O.rhs_vjp(m, y, mt, fb)
    meta = np.array([mt], np.int32)

    def L(yy, model=m):
        return float(fb @ O.rhs(model, yy[None], meta)[0])

    for trial in range(3):
        v = rng.normal(size=48)
        v[live:] = 0
        e = 1e-6
        fd = (L(y + e * v) - L(y - e * v)) / (2 * e)
        assert abs(fd - yb @ v) <= 1e-9 * np.linalg.norm(yb) * np.linalg.norm(v), (trial, fd, yb @ v)
    G, Gb = (gs, gsb) if cls >= 2 else (gp, gpb)
    other = gp if cls >= 2 else gs
    assert not np.any(gsb if cls < 2 else gpb)   # the other wave's grid is not read
    base = tuple(int(t) for t in np.clip(np.floor(y[0:3] / h), 0, gp.shape[0] - 2))
    for corner in [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]:
        nd = tuple(i + c for i, c in zip(base, corner))
        for f in range(10):
            step = 2.0 ** -12
            Gp_, Gm_ = G.copy(), G.copy()
            Gp_[nd + (f,)] += np.float32(step)
            Gm_[nd + (f,)] -= np.float32(step)
            mk = (lambda GG: O.Model("grid", grid_p=other, grid_s=GG, spacing=(h, h, h))) if cls >= 2 else \
                (lambda GG: O.Model("grid", grid_p=GG, grid_s=other, spacing=(h, h, h)))
            fd = (L(y, mk(Gp_)) - L(y, mk(Gm_))) / (2 * step)
            assert abs(fd - Gb[nd + (f,)]) <= 1e-7 * max(abs(fd), 1e-3), (nd, f, fd, Gb[nd + (f,)])


def _small_problem(O, with_g=True, interior=True):
    k = 16.0
    gp, gs, h = _grid()
    x0 = np.array([0.31, 0.47, 0.52])
    d = np.array([1.0, 0.0, 0.0])
    b = np.array([0.2, -0.5, 1.0])
    b /= np.linalg.norm(b)
    ny = 24
    y0, dy = W._ygrid(x0, W.window_radius(k), ny)
    f = W._packet(y0, dy, ny, k, x0, b, d)
    g = 0.3j * f if with_g else None
    mesh = oracle_mesh(O, W.centred_mesh(3, x0, 3, d, W.mesh_radius(k, 6.0), W.mesh_radius(k, 4.8)))
    F = O.fbi(f, y0, dy, k, mesh)
    G = O.fbi(g, y0, dy, k, mesh) if with_g else None
    r = (np.arange(4) + 0.5) / 4
    R1, R2 = np.meshgrid(r, r, indexing="ij")
    rx = np.stack([np.full(R1.size, 0.7), R1.ravel(), R2.ravel()], -1)
    times = np.array([0.033, 0.1, 0.151, 0.2]) if interior else np.array([0.05, 0.1, 0.15, 0.2])
    return dict(k=k, gp=gp, gs=gs, h=h, mesh=mesh, F=F, G=G, rx=rx, dt=0.01, nsteps=20, times=times,
                rw=W.window_radius(k))


def _misfit(O, P, a, b, dobs, classes=(0, 1, 2, 3)):
    h = P["h"]
    m = O.Model("grid", grid_p=a, grid_s=b, spacing=(h, h, h))
    u = O.solve(m, P["k"], P["mesh"], P["F"], P["G"], classes, P["dt"], P["nsteps"], P["times"], P["rx"], P["rw"])
    return 0.5 * float(np.sum(np.abs(u - dobs) ** 2)), u, m


@pytest.fixture(scope="module")
def problem(oracle):
    O = oracle
    P = _small_problem(O)
    dobs = O.solve(O.Model("grid", grid_p=P["gp"] * np.float32(1.01), grid_s=P["gs"] * np.float32(0.99),
                           spacing=(P["h"],) * 3), P["k"], P["mesh"], P["F"], P["G"], (0, 1, 2, 3), P["dt"],
                   P["nsteps"], P["times"], P["rx"], P["rw"])
    L0, u0, m = _misfit(O, P, P["gp"], P["gs"], dobs)
    gpb, gsb = O.solve_vjp(m, P["k"], P["mesh"], P["F"], P["G"], (0, 1, 2, 3), P["dt"], P["nsteps"], P["times"],
                           P["rx"], P["rw"], u0 - dobs)
    return P, dobs, gpb, gsb


def test_solve_vjp_single_entries(oracle, problem):
    O = oracle
    P, dobs, gpb, gsb = problem
    inner = np.zeros(gpb.shape, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    step = 2.0 ** -14
    for G, Gb, wave in ((P["gp"], gpb, 0), (P["gs"], gsb, 1)):
        order = np.argsort(-np.abs(np.where(inner, Gb, 0)).reshape(-1))
        picks = list(order[:4]) + list(order[20:22])
        for flat in picks:
            nd = np.unravel_index(flat, Gb.shape)
            A, B = G.copy(), G.copy()
            A[nd] += np.float32(step)
            B[nd] -= np.float32(step)
            if wave == 0:
                fd = (_misfit(O, P, A, P["gs"], dobs)[0] - _misfit(O, P, B, P["gs"], dobs)[0]) / (2 * step)
            else:
                fd = (_misfit(O, P, P["gp"], A, dobs)[0] - _misfit(O, P, P["gp"], B, dobs)[0]) / (2 * step)
            assert abs(fd - Gb[nd]) <= 1e-6 * abs(Gb[nd]) + 1e-12, (wave, nd, fd, Gb[nd])


def test_solve_vjp_random_directions(oracle, problem):
    O = oracle
    P, dobs, gpb, gsb = problem
    rng = np.random.default_rng(3)
    for trial in range(2):
        Vp = rng.normal(size=gpb.shape)
        Vs = rng.normal(size=gsb.shape)
        eps = 1e-4
        ap, am = (P["gp"] + eps * Vp).astype(np.float32), (P["gp"] - eps * Vp).astype(np.float32)
        bp, bm = (P["gs"] + eps * Vs).astype(np.float32), (P["gs"] - eps * Vs).astype(np.float32)
        fd = _misfit(O, P, ap, bp, dobs)[0] - _misfit(O, P, am, bm, dobs)[0]
        lin = float(np.sum(gpb * (ap.astype(np.float64) - am)) + np.sum(gsb * (bp.astype(np.float64) - bm)))
        # beams crossing cell faces inside +-eps leave a small kink term
        assert abs(fd - lin) <= 2e-5 * abs(fd), (trial, fd, lin)


def test_init_vjp_term(oracle):
    """With a velocity term the initial amplitudes depend on c(q): dropping that term (solve_vjp
    without the initial-velocity data is a different problem) must change the gradient, and the
    full gradient still matches differences at the mesh's q nodes' neighbourhood."""
    O = oracle
    P = _small_problem(O, with_g=True, interior=False)
    Pn = _small_problem(O, with_g=False, interior=False)
    dobs = np.zeros((len(P["times"]), P["rx"].shape[0], 3), complex)
    _, u0, m = _misfit(O, P, P["gp"], P["gs"], dobs, classes=(0,))
    gpb, _ = O.solve_vjp(m, P["k"], P["mesh"], P["F"], P["G"], (0,), P["dt"], P["nsteps"], P["times"], P["rx"],
                         P["rw"], u0)
    _, u1, m1 = _misfit(O, Pn, Pn["gp"], Pn["gs"], dobs, classes=(0,))
    gpn, _ = O.solve_vjp(m1, Pn["k"], Pn["mesh"], Pn["F"], None, (0,), Pn["dt"], Pn["nsteps"], Pn["times"],
                         Pn["rx"], Pn["rw"], u1)
    assert np.linalg.norm(gpb - gpn) > 1e-3 * np.linalg.norm(gpb)
    # the c field at the node nearest the source, where the initial amplitudes sample c(q)
    nd = (2, 4, 4, 0)
    step = 2.0 ** -14
    A, B = P["gp"].copy(), P["gp"].copy()
    A[nd] += np.float32(step)
    B[nd] -= np.float32(step)
    fd = (_misfit(O, P, A, P["gs"], dobs, (0,))[0] - _misfit(O, P, B, P["gs"], dobs, (0,))[0]) / (2 * step)
    assert abs(fd - gpb[nd]) <= 1e-6 * abs(gpb[nd]), (fd, gpb[nd])
