"""Discrete adjoint on the GPU (fga_solve_vjp) against the oracle's reverse mode, against finite
differences of the GPU's own forward map, and through torch.autograd.

Problem: the crosswell geometry at a reduced size (k = 16, 9^3 model grid, one source off the grid
planes with an initial-velocity term, 3^3 x 3^3 mesh per class, 20 RK4 steps, samples inside and at
the end of steps, 16 receivers); the observed data come from the oracle on the true (bumped) model.
"""
import math

import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup, oracle_beams, oracle_model, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu

# The FP64 and FP32 bars of the forward path (relative L2 1e-10 and 1e-4 against the FP64 oracle).
# Measured on GB300: FP64 2e-15 (same discrete map, different summation order), FP32 2e-5 (the FP32
# rounding of the trajectory, amplified by k |x - Q| in the phase derivatives).
TOL = {1: 1e-10, 0: 1e-4}


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _problem(v0=0.3j, times=(0.033, 0.1, 0.151, 0.2)):
    ws, true = W.crosswell(n_src_side=1, nq=3, np_=3, ny=24, nsteps=20, dt=0.01, k=16.0, grid_n=9, rx_side=4,
                           times=list(times), v0=v0, src_x1=0.31, src_offset=(-0.03, 0.02))
    return ws[0], true


@pytest.fixture(scope="module")
def oracle_case(oracle):
    O = oracle
    w, true = _problem()
    model = oracle_model(O, w.medium)
    mesh = oracle_mesh(O, w.mesh)
    F = O.fbi(w.f, w.y0, w.dy, w.k, mesh)
    G = O.fbi(w.g, w.y0, w.dy, w.k, mesh)
    args = (w.k, mesh, F, G, w.classes, w.dt, w.nsteps, w.times, w.receivers, w.rw)
    d = O.solve(oracle_model(O, true), *args)
    u = O.solve(model, *args)
    ub = u - d
    gp, gs = O.solve_vjp(model, *args, ub)
    return w, true, ub, gp, gs


def _gpu_grads(fga, w, ub, prec, checkpoint_every=20):
    import torch
    model, desc, keep = gpu_setup(w, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    cdt = torch.complex128 if prec == 1 else torch.complex64
    ubar = torch.as_tensor(ub, device="cuda").to(cdt)
    gp, gs = fga.solve_vjp(model, desc, w.dt, w.nsteps, w.times, rx, ubar, rw=w.rw,
                           checkpoint_every=checkpoint_every)
    torch.cuda.synchronize()
    return gp.cpu().numpy(), gs.cpu().numpy()


@pytest.mark.parametrize("prec", [1, 0])
def test_vjp_matches_oracle(fga, oracle_case, prec):
    w, true, ub, ogp, ogs = oracle_case
    gp, gs = _gpu_grads(fga, w, ub, prec)
    assert np.linalg.norm(ogp) > 0 and np.linalg.norm(ogs) > 0
    assert rel_l2(gp, ogp) <= TOL[prec], rel_l2(gp, ogp)
    assert rel_l2(gs, ogs) <= TOL[prec], rel_l2(gs, ogs)


@pytest.mark.parametrize("every", [1, 7, 20, 50])
def test_checkpoint_interval_does_not_change_gradient(fga, oracle_case, every):
    w, true, ub, ogp, ogs = oracle_case
    gp, gs = _gpu_grads(fga, w, ub, 1, every)
    ref_p, ref_s = _gpu_grads(fga, w, ub, 1, 20)
    assert rel_l2(gp, ref_p) <= 1e-13 and rel_l2(gs, ref_s) <= 1e-13


def test_vjp_matches_gpu_differences(fga, oracle_case):
    """dL/d(grid entry) from the GPU adjoint equals central differences of the GPU's own FP64 forward."""
    import torch
    w, true, ub, ogp, ogs = oracle_case
    rx = torch.as_tensor(w.receivers, device="cuda")
    model0, desc, keep = gpu_setup(w, 1)
    u0, _ = fga.solve(model0, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    d = u0 - torch.as_tensor(ub, device="cuda")   # observed data such that u0 - d = ub
    gp, gs = fga.solve_vjp(model0, desc, w.dt, w.nsteps, w.times, rx, u0 - d, rw=w.rw)
    gp, gs = gp.cpu().numpy(), gs.cpu().numpy()
    h = w.medium.spacing

    def L(grid_p, grid_s):
        m = fga.Model("grid", grid_p=torch.as_tensor(grid_p, device="cuda"),
                      grid_s=torch.as_tensor(grid_s, device="cuda"), origin=w.medium.origin, spacing=h)
        u, _ = fga.solve(m, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
        return 0.5 * float((u - d).abs().pow(2).sum())

    step = 2.0 ** -14
    inner = np.zeros(gp.shape, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    for wave, (G, Gb) in enumerate(((w.medium.grid_p, gp), (w.medium.grid_s, gs))):
        for flat in np.argsort(-np.abs(np.where(inner, Gb, 0)).reshape(-1))[:3]:
            nd = np.unravel_index(flat, Gb.shape)
            A, B = G.copy(), G.copy()
            A[nd] += np.float32(step)
            B[nd] -= np.float32(step)
            if wave == 0:
                fd = (L(A, w.medium.grid_s) - L(B, w.medium.grid_s)) / (2 * step)
            else:
                fd = (L(w.medium.grid_p, A) - L(w.medium.grid_p, B)) / (2 * step)
            assert abs(fd - Gb[nd]) <= 1e-6 * abs(Gb[nd]), (wave, nd, fd, Gb[nd])


def test_autograd_through_node_speeds(fga, oracle_case):
    """torch.autograd: L(c_p nodes) with fields by finite differences and c_s = c_p/sqrt(3); the
    gradient w.r.t. c_p nodes matches a central difference of the whole pipeline."""
    import torch
    from paper_1810_06760_gb300 import adjoint as A
    w, true, ub, ogp, ogs = oracle_case
    model, desc, keep = gpu_setup(w, 1)
    rx = torch.as_tensor(w.receivers, device="cuda")
    n = w.medium.grid_p.shape[0]
    h = w.medium.spacing[0]
    cp0 = torch.as_tensor(w.medium.grid_p[..., 0].astype(np.float64), device="cuda")
    spec = A.SourceSpec(desc, w.dt, w.nsteps, np.asarray(w.times), rx, rw=w.rw, origin=w.medium.origin,
                        spacing=w.medium.spacing, keep=keep)
    fp_true = torch.as_tensor(true.grid_p, device="cuda")
    fs_true = torch.as_tensor(true.grid_s, device="cuda")
    d = A.seismograms(fp_true, fs_true, spec).detach()

    def loss(cp):
        fp = A.fields_from_nodes(cp, h)
        fs = A.fields_from_nodes(A.cs_from_cp(cp), h)
        return A.misfit(A.seismograms(fp.float(), fs.float(), spec), d)

    cp = cp0.clone().requires_grad_(True)
    Lv = loss(cp)
    Lv.backward()
    g = cp.grad.cpu().numpy()
    assert np.isfinite(g).all() and np.abs(g).max() > 0
    for flat in np.argsort(-np.abs(g[1:-1, 1:-1, 1:-1]).reshape(-1))[:3]:
        i = np.unravel_index(flat, (n - 2,) * 3)
        nd = tuple(int(v) + 1 for v in i)
        e = 2.0 ** -9
        with torch.no_grad():
            cpp, cpm = cp0.clone(), cp0.clone()
            cpp[nd] += e
            cpm[nd] -= e
            fd = (float(loss(cpp)) - float(loss(cpm))) / (2 * e)
        # the fields are rounded to FP32 for the model grids: the difference carries ~1e-4 of that rounding
        assert abs(fd - g[nd]) <= 2e-3 * abs(g[nd]), (nd, fd, g[nd])


def test_vjp_constant_medium_and_errors(fga):
    import torch
    w = W.homogeneous(nq=3, np_=3, ny=24, nsteps=10, dt=0.01, n_receivers=8, k=16.0, n_times=2)
    model, desc, keep = gpu_setup(w, 1)
    rx = torch.as_tensor(w.receivers, device="cuda")
    ub = torch.ones((2, 8, 3), dtype=torch.complex128, device="cuda")
    assert fga.solve_vjp(model, desc, w.dt, w.nsteps, w.times, rx, ub) == (None, None)
    with pytest.raises(fga.FGAError) as e:
        fga.solve_vjp(model, desc, w.dt, w.nsteps, np.linspace(0.001, 0.0019, 5) + 0.05, rx,
                      torch.ones((5, 8, 3), dtype=torch.complex128, device="cuda"))
    assert e.value.status != 0
    lw = W.layered(nq=2, np_=2, ny=16, nsteps=4, dt=0.1, n_times=2, rx_side=2)
    lm, ld, lk = gpu_setup(lw, 1)
    lrx = torch.as_tensor(lw.receivers, device="cuda")
    with pytest.raises(fga.FGAError):
        fga.solve_vjp(lm, ld, lw.dt, lw.nsteps, lw.times, lrx,
                      torch.ones((2, lrx.shape[0], 3), dtype=torch.complex128, device="cuda"))


def test_vjp_32_seeded_cells(fga, oracle_case):
    """Central differences of the GPU FP64 forward at 32 grid entries drawn with rng seed 2 (among the
    interior entries whose gradient is not negligible) agree with the adjoint to 1e-5."""
    import torch
    w, true, ub, ogp, ogs = oracle_case
    rx = torch.as_tensor(w.receivers, device="cuda")
    model0, desc, keep = gpu_setup(w, 1)
    u0, _ = fga.solve(model0, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    d = u0 - torch.as_tensor(ub, device="cuda")
    gp, gs = fga.solve_vjp(model0, desc, w.dt, w.nsteps, w.times, rx, u0 - d, rw=w.rw)
    grads = (gp.cpu().numpy(), gs.cpu().numpy())
    grids = (w.medium.grid_p, w.medium.grid_s)

    def L(grid_p, grid_s):
        m = fga.Model("grid", grid_p=torch.as_tensor(grid_p, device="cuda"),
                      grid_s=torch.as_tensor(grid_s, device="cuda"), origin=w.medium.origin, spacing=w.medium.spacing)
        u, _ = fga.solve(m, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
        return 0.5 * float((u - d).abs().pow(2).sum())

    cands = []
    for wave in (0, 1):
        G = grads[wave]
        inner = np.zeros(G.shape, bool)
        inner[1:-1, 1:-1, 1:-1] = True
        ok = inner & (np.abs(G) > 1e-3 * np.abs(G).max())
        cands += [(wave, tuple(int(v) for v in ix)) for ix in np.argwhere(ok)]
    rng = np.random.default_rng(2)
    picks = rng.choice(len(cands), size=min(32, len(cands)), replace=False)
    step = 2.0 ** -14
    errs = []
    for pi in picks:
        wave, nd = cands[pi]
        A, B = grids[wave].copy(), grids[wave].copy()
        A[nd] += np.float32(step)
        B[nd] -= np.float32(step)
        if wave == 0:
            fd = (L(A, grids[1]) - L(B, grids[1])) / (2 * step)
        else:
            fd = (L(grids[0], A) - L(grids[0], B)) / (2 * step)
        errs.append(abs(fd - grads[wave][nd]) / abs(grads[wave][nd]))
    assert len(errs) == 32 and max(errs) <= 1e-5, max(errs)


def test_vjp_releases_device_memory(fga):
    """Repeated adjoint calls return their checkpoint and segment storage."""
    import torch
    ws, true = W.crosswell(n_src_side=1, nq=6, np_=6, ny=32, nsteps=40, dt=0.005, k=32.0, grid_n=17, rx_side=4,
                           n_times=10)
    w = ws[0]
    model, desc, keep = gpu_setup(w, 0)
    rx = torch.as_tensor(w.receivers, device="cuda")
    u, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    gp, gs = fga.solve_vjp(model, desc, w.dt, w.nsteps, w.times, rx, u)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        fga.solve_vjp(model, desc, w.dt, w.nsteps, w.times, rx, u, grad_p=gp, grad_s=gs)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # one call holds (ceil(40/20) + 20 + 2) x 46 x 4 B per beam ~ 160 MB; five leaked calls would lose 800 MB
    assert free0 - free1 < 64 * 2 ** 20, (free0 - free1) / 2 ** 20
