"""Beam selection of step 1 of Fig. fig:FGA_alg (only the beams with |psi| > eps max|psi| are created),
through the C ABI, against the oracle's selection (itself pinned to the closed-form survivors of a
Gaussian packet).

Which beams survive is index work and is compared exactly, except for the beams whose |psi|/max|psi|
lies so close to eps that the two precisions may decide differently: within 2e-5 (FP32: the
transform's absolute error is a few 1e-6 of the largest value) or 1e-11 (FP64) of eps.  Those may go
either way.  The states of the beams both sides keep are compared at the usual bars (relative L2
1e-4 FP32, 1e-10 FP64), and a whole solve on the selected set is compared with the oracle's sum over
the same set, so class blocks whose sizes are not multiples of the mesh size go through propagation,
records and the Gaussian sum."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup, max_rel_dominant, oracle_beams, rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}
AMBIG = {0: 2e-5, 1: 1e-11}


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _work(**kw):
    args = dict(nq=6, np_=4, ny=24, nsteps=24, n_samples=12, rx_side=6, snap_side=0, grid_n=33, grid=False)
    args.update(kw)
    return W.smooth(**args)


def _oracle_selection(oracle, w, eps):
    omodel, mesh, obeams = oracle_beams(oracle, w)
    groups = [(st, mt) for _, st, mt in obeams]
    mags = [np.sqrt(np.sum(np.abs(oracle.state_a(st)) ** 2, axis=1)) for st, _ in groups]
    top = max(m.max() for m in mags)
    return omodel, mesh, obeams, oracle.psi_select(groups, eps), [m / top for m in mags]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("eps", [3e-1, 1e-2, 1e-4])
def test_selection_matches_oracle(fga, oracle, prec, eps):
    w = _work()
    model, desc, keep = gpu_setup(w, prec)
    desc.psi_rel_min = eps
    beams = fga.decompose(model, desc)
    st, meta, mid, _, _ = beams.export_all()
    beams.close()
    _, _, obeams, sel, ratio = _oracle_selection(oracle, w, eps)
    n_total = 0
    for i, (cls, ost, _) in enumerate(obeams):
        g = (meta & 3) == cls
        gids = mid[g]
        assert np.all(np.diff(gids) > 0)                       # mesh order within the class block
        clear = np.abs(ratio[i] - eps) > AMBIG[prec]
        want = set(np.nonzero((ratio[i] > eps) & clear)[0])
        got = set(gids.tolist()) & set(np.nonzero(clear)[0])
        assert got == want, (cls, len(got), len(want))
        common, gi, oi = np.intersect1d(gids, sel[i][2], return_indices=True)
        assert common.size > 0
        gs = st[g][gi]
        os_ = ost[common]
        for sl in (slice(0, 6), slice(6, 42), slice(42, 46)):
            assert rel_l2(gs[:, sl], os_[:, sl]) <= TOL[prec], (cls, sl)
        n_total += g.sum()
    assert n_total == len(meta)
    assert n_total < len(obeams) * w.mesh.M                  # the selection dropped beams


@pytest.mark.parametrize("prec", [1, 0])
def test_solve_on_selected_beams(fga, oracle, prec):
    """fga_solve with psi_rel_min: seismograms against the oracle's sum over its own selected beams."""
    import torch
    eps = 1e-2
    w = _work()
    model, desc, keep = gpu_setup(w, prec)
    desc.psi_rel_min = eps
    rx = torch.as_tensor(w.receivers, device="cuda")
    seis, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    torch.cuda.synchronize()
    omodel, mesh, obeams, sel, ratio = _oracle_selection(oracle, w, eps)
    amb = [np.abs(r - eps) <= AMBIG[prec] for r in ratio]
    assert not any(a.any() for a in amb), "a beam sits on the threshold; pick another eps"
    wgt = mesh.weight(w.k)
    s_step, s_th = oracle.sample_schedule(w.times, w.dt, w.nsteps)
    ref = np.zeros((len(w.times), len(w.receivers), 3), complex)
    for (cls, _, _), (st, mt, _) in zip(obeams, sel):
        st = st.copy()
        rec = oracle.propagate(omodel, st, mt, w.dt, w.nsteps, s_step, s_th, wgt)
        for j in range(len(w.times)):
            ref[j] += oracle.gauss_sum(rec[j], w.k, w.rw, w.receivers)
    got = seis.cpu().numpy()
    assert np.abs(ref).max() > 0
    assert rel_l2(got, ref) <= TOL[prec], rel_l2(got, ref)
    assert max_rel_dominant(got, ref, 1e-2) <= (2e-3 if prec == 0 else 1e-9)


def test_selection_of_zero_data_is_empty(fga):
    """All-zero initial data: no beam exceeds eps x 0, the set is empty, and a solve returns zeros."""
    import torch
    w = _work()
    model, desc, keep = gpu_setup(w, 0)
    z = torch.zeros_like(keep[0])
    desc.f = z.data_ptr()
    desc.psi_rel_min = 1e-3
    beams = fga.decompose(model, desc)
    assert int(beams.count().sum()) == 0
    beams.close()
    rx = torch.as_tensor(w.receivers, device="cuda")
    seis, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    torch.cuda.synchronize()
    assert float(seis.abs().max()) == 0.0


def test_selection_rejections(fga):
    """psi_rel_min outside [0, 1) is rejected, and so is a selection given to the adjoint."""
    import torch
    w = _work()
    model, desc, keep = gpu_setup(w, 0)
    for bad in (-1e-3, 1.0, float("nan")):
        desc.psi_rel_min = bad
        with pytest.raises(fga.FGAError):
            fga.decompose(model, desc)
    desc.psi_rel_min = 1e-3
    rx = torch.as_tensor(w.receivers, device="cuda")
    ubar = torch.zeros((len(w.times), len(w.receivers), 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(fga.FGAError) as e:
        fga.solve_vjp(model, desc, w.dt, w.nsteps, w.times, rx, ubar, rw=w.rw)
    assert e.value.status == fga.FGA_ERR_INVALID_ARG
