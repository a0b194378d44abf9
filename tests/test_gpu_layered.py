"""Layered media (Sec. 3.1) on the GPU against the oracle: beams split at flat interfaces into
reflected and transmitted P and S children; the populations are matched by lineage (mesh point and
path of child slots) and compared state by state, then the seismograms at step-end samples."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup, max_rel_dominant, oracle_beams, oracle_model, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}
GROUPS = {"Q": slice(0, 3), "P": slice(3, 6), "dzQ": slice(6, 24), "dzP": slice(24, 42), "a": slice(42, 46)}


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _oracle_population(O, w, nsteps, gmax=4, rel_min=1e-6):
    omodel, mesh, obeams = oracle_beams(O, w)
    st = np.concatenate([b[1] for b in obeams])
    meta = np.concatenate([b[2] for b in obeams])
    mid = np.concatenate([np.arange(b[1].shape[0]) for b in obeams])
    path = np.zeros(st.shape[0], dtype=np.int64)
    for _ in range(nsteps):
        st, meta, path, parent = O.layered_step(omodel, st, meta, path, w.dt, gmax, rel_min, return_parent=True)
        mid = mid[parent]
    return st, meta, mid, path


def _key(meta, mid, path):
    # lineage: class of the initial beam (meta bits 13-14), its mesh point, the path of child slots
    return [((int(m) >> 13) & 3, int(i), int(p)) for m, i, p in zip(meta, mid, path)]


@pytest.mark.parametrize("prec", [1, 0])
def test_layered_population_matches_oracle(fga, oracle, prec):
    w = W.layered(nq=3, np_=4, ny=24, nsteps=30, dt=0.1)
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    gst, gmeta, gmid, gpath, dropped = beams.export_all()
    ost, ometa, omid, opath = _oracle_population(oracle, w, w.nsteps)
    assert dropped == 0
    gk, ok = _key(gmeta, gmid, gpath), _key(ometa, omid, opath)
    assert len(set(ok)) == len(ok) and len(set(gk)) == len(gk)
    common = sorted(set(gk) & set(ok))
    # events decided in FP32 may differ from FP64 for a beam ending a step within rounding of an interface
    need = 1.0 if prec == 1 else 0.999
    assert len(common) >= need * len(ok) and len(common) >= need * len(gk), (len(common), len(ok), len(gk))
    assert len(ok) > 1.5 * (w.n_beams)      # interfaces were really crossed
    gi = {k: i for i, k in enumerate(gk)}
    oi = {k: i for i, k in enumerate(ok)}
    G = np.stack([gst[gi[k]] for k in common])
    Ob = np.stack([ost[oi[k]] for k in common])
    np.testing.assert_array_equal(np.array([gmeta[gi[k]] for k in common]) & 0x6FF7,
                                  np.array([ometa[oi[k]] for k in common]) & 0x6FF7)
    for name, sl in GROUPS.items():
        assert rel_l2(G[:, sl], Ob[:, sl]) <= TOL[prec], name


@pytest.mark.parametrize("prec", [1, 0])
def test_layered_solve_seismograms(fga, oracle, prec):
    import torch
    w = W.layered(nq=3, np_=4, ny=24, nsteps=24, dt=0.1, n_times=6, rx_side=6)
    model, desc, keep = gpu_setup(w, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    seis, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    torch.cuda.synchronize()
    omodel = oracle_model(oracle, w.medium)
    mesh = oracle_mesh(oracle, w.mesh)
    wgt = mesh.weight(w.k)
    omodel, mesh, obeams = oracle_beams(oracle, w)
    st = np.concatenate([b[1] for b in obeams])
    meta = np.concatenate([b[2] for b in obeams])
    path = np.zeros(st.shape[0], dtype=np.int64)
    ref = np.zeros((len(w.times), rx.shape[0], 3), complex)
    j = 0
    for n in range(1, w.nsteps + 1):
        st, meta, path = oracle.layered_step(omodel, st, meta, path, w.dt)
        while j < len(w.times) and abs(w.times[j] - n * w.dt) < 1e-9:
            ref[j] = oracle.gauss_sum(oracle.records(st, meta, wgt), w.k, w.rw, w.receivers)
            j += 1
    # the oracle's interface events follow the printed Zoeppritz system, the library's the 6 x 6
    # continuity solve; on this case every lineage matches and FP32 stays near 4e-6
    assert rel_l2(seis.cpu().numpy(), ref) <= TOL[prec]
    assert max_rel_dominant(seis.cpu().numpy(), ref, 1e-2) <= (2e-3 if prec == 0 else 1e-9)
