"""Serving loop (fga_server_*): requests of different k, mesh sizes and sources on one resident model.
A request's seismograms are bit-identical whether it runs alone (fga_solve) or among others; the
admission budget bounds concurrency; a failing request reports its own error and the server keeps
serving; a bounded wait times out without losing the request."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _requests():
    return W.serving_requests(n=6, seed=3, n_range=(2e3, 6e4), ks=(16.0, 32.0), np_=4, nsteps=12, dt=0.01,
                              rx_side=4, n_times=6, grid_n=32)


@pytest.mark.parametrize("prec", [0, 1])
def test_results_identical_alone_and_in_mix(fga, prec):
    import torch
    reqs = _requests()
    w0 = reqs[0].workload
    model = fga.model_from_medium(w0.medium)
    alone = []
    lattice = prec == 0   # FP32 requests take their receivers as a lattice, FP64 ones as points
    for r in reqs:
        w = r.workload
        _, desc, k = gpu_setup(w, prec)
        rx = torch.as_tensor(w.receivers, device="cuda")
        if lattice:
            u, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rw=w.rw, rx_axes=w.rx_axes)
        else:
            u, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
        torch.cuda.synchronize()
        alone.append(u.cpu())
    server = fga.Server(model, n_workers=3)
    ids = []
    keep = []
    for r in reqs:
        w = r.workload
        _, desc, k = gpu_setup(w, prec)
        rx = torch.as_tensor(w.receivers, device="cuda")
        if lattice:
            ids.append(server.submit(desc, w.dt, w.nsteps, w.times, rw=w.rw, keep=k, rx_axes=w.rx_axes))
        else:
            ids.append(server.submit(desc, w.dt, w.nsteps, w.times, rx, rw=w.rw, keep=k))
    infos = []
    for i, rid in enumerate(ids):
        u, info = server.wait(rid)
        infos.append(info)
        assert torch.equal(u.cpu(), alone[i]), i
        assert info["t_submit"] <= info["t_start"] <= info["t_end"]
        assert info["beams"] == reqs[i].workload.n_beams
    st = server.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["running"] == 0
    assert 1 <= st["peak_running"] <= 3
    server.close()


def test_budget_serialises_and_errors_are_per_request(fga):
    import torch
    reqs = _requests()
    model = fga.model_from_medium(reqs[0].workload.medium)
    server = fga.Server(model, n_workers=4, hbm_budget_bytes=1.0)   # every request exceeds it alone
    ids, keep = [], []
    for j, r in enumerate(reqs[:4]):
        w = r.workload
        _, desc, k = gpu_setup(w, 0)
        rx = torch.as_tensor(w.receivers, device="cuda")
        times = w.times if j != 1 else np.array([w.T * 2.0])     # request 1: a sample after the end
        ids.append(server.submit(desc, w.dt, w.nsteps, times, rx, rw=w.rw, keep=k))
    spans = []
    for j, rid in enumerate(ids):
        if j == 1:
            with pytest.raises(fga.FGAError) as e:
                server.wait(rid)
            assert e.value.status == 1 and "sample times" in str(e.value)
            continue
        u, info = server.wait(rid)
        assert torch.isfinite(torch.view_as_real(u)).all()
        spans.append((info["t_start"], info["t_end"]))
    st = server.stats()
    assert st["peak_running"] == 1
    spans.sort()
    for a, b in zip(spans, spans[1:]):
        assert a[1] <= b[0]     # no overlap under a budget that admits one request at a time
    server.close()


def test_wait_timeout_keeps_request(fga):
    import torch
    reqs = W.serving_requests(n=1, seed=5, n_range=(2e5, 2e5), ks=(32.0,), np_=8, nsteps=60, dt=0.005,
                              rx_side=8, n_times=60, grid_n=32)
    w = reqs[0].workload
    model = fga.model_from_medium(w.medium)
    server = fga.Server(model, n_workers=1)
    _, desc, k = gpu_setup(w, 0)
    rx = torch.as_tensor(w.receivers, device="cuda")
    rid = server.submit(desc, w.dt, w.nsteps, w.times, rx, rw=w.rw, keep=k)
    with pytest.raises(fga.FGAError) as e:
        server.wait(rid, timeout=1e-6)
    assert e.value.status == 4
    u, info = server.wait(rid)
    assert u.shape == (w.times.size, rx.shape[0], 3)
    server.close()
