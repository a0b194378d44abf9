"""Reconstruction at points given in spherical coordinates (Sec. 3: only the reconstruction point x of
Eq. FGA changes; decomposition and propagation are coordinate free), through the C ABI: against the
oracle's brute-force sum at the converted points, against the library's own Cartesian call, and inside
a whole solve."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup, max_rel_dominant, oracle_beams, rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _rtp(n, seed):
    """Points on shells around the origin that fall inside the smooth workload's box [0, 1]^3."""
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(0.35, 1.2, n), rng.uniform(0.05, 1.5, n), rng.uniform(0.05, 1.2, n)], -1)


def _small():
    return W.smooth(nq=5, np_=3, ny=24, nsteps=16, n_samples=6, rx_side=4, snap_side=0, grid_n=33)


@pytest.mark.parametrize("prec", [1, 0])
def test_reconstruct_spherical_matches_oracle(fga, oracle, prec):
    import torch
    w = _small()
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    rtp = _rtp(101, 3)
    u = fga.reconstruct_spherical(beams, torch.as_tensor(rtp, device="cuda"), rw=w.rw).cpu().numpy()
    x = oracle.spherical_to_cartesian(rtp)
    omodel, mesh, obeams = oracle_beams(oracle, w)
    ref = np.zeros((x.shape[0], 3), complex)
    for cls, st, meta in obeams:
        oracle.propagate(omodel, st, meta, w.dt, w.nsteps)
        ref += oracle.gauss_sum(oracle.records(st, meta, mesh.weight(w.k)), w.k, w.rw, x)
    assert rel_l2(u, ref) <= TOL[prec]
    assert max_rel_dominant(u, ref, 1e-2) <= (2e-3 if prec == 0 else 1e-9)
    # the same as the Cartesian call at the converted points
    uc = fga.reconstruct(beams, torch.as_tensor(x, device="cuda"), rw=w.rw).cpu().numpy()
    assert rel_l2(u, uc) <= (1e-6 if prec == 0 else 1e-13)


@pytest.mark.parametrize("prec", [1, 0])
def test_solve_with_spherical_receivers(fga, prec):
    """A solve whose receivers are (r, theta, phi) gives the seismograms of the same receivers given in
    Cartesian coordinates."""
    import torch
    w = _small()
    model, desc, keep = gpu_setup(w, prec)
    rtp = _rtp(37, 4)
    x = np.stack([rtp[:, 0] * np.cos(rtp[:, 1]) * np.cos(rtp[:, 2]), rtp[:, 0] * np.sin(rtp[:, 1]) * np.cos(rtp[:, 2]),
                  rtp[:, 0] * np.sin(rtp[:, 2])], -1)
    s1, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, torch.as_tensor(rtp, device="cuda"), rw=w.rw,
                      spherical=True)
    s2, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, torch.as_tensor(x, device="cuda"), rw=w.rw)
    torch.cuda.synchronize()
    assert rel_l2(s1.cpu().numpy(), s2.cpu().numpy()) <= (1e-6 if prec == 0 else 1e-13)
    assert float(s2.abs().max()) > 0
    with pytest.raises(fga.FGAError):      # lattices are Cartesian only
        fga.solve(model, desc, w.dt, w.nsteps, w.times, rw=w.rw, rx_axes=w.rx_axes, spherical=True)
