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


def _blocker(n_steps=400):
    """A request that keeps one worker busy for many windows of steps (a few hundred milliseconds)."""
    return W.serving_requests(n=1, seed=7, n_range=(3e5, 3e5), ks=(32.0,), np_=8, nsteps=n_steps, dt=0.0025,
                              rx_side=8, n_times=n_steps, grid_n=32)[0].workload


def _submit(fga, server, w, prec=0):
    import torch
    _, desc, k = gpu_setup(w, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    return server.submit(desc, w.dt, w.nsteps, w.times, rx, rw=w.rw, keep=k)


@pytest.mark.parametrize("policy,age", [(1, 0.0), (1, 1e-6), (0, 0.0)])
def test_admission_order(fga, policy, age):
    """One worker, busy with a long request while three more are queued (large, small, medium): the
    shortest-estimated-work policy starts the small one first; with an age limit that every waiting
    request exceeds, and with FIFO, they start in submission order."""
    blocker = _blocker()
    model = fga.model_from_medium(blocker.medium)
    server = fga.Server(model, n_workers=1, policy=policy, age_limit_s=age)
    first = _submit(fga, server, blocker)
    sizes = {"large": 6e4, "small": 2e3, "medium": 2e4}
    ids = {}
    for name, n in sizes.items():
        w = W.serving_requests(n=1, seed=3, n_range=(n, n), ks=(16.0,), np_=4, nsteps=12, dt=0.01, rx_side=4,
                               n_times=6, grid_n=32)[0].workload
        ids[name] = _submit(fga, server, w)
    server.wait(first)
    starts = {name: server.wait(rid)[1]["t_start"] for name, rid in ids.items()}
    order = sorted(starts, key=lambda n: starts[n])
    if policy == 1 and age == 0.0:
        assert order == ["small", "medium", "large"], starts
    else:
        assert order == ["large", "small", "medium"], starts
    server.close()


def test_cancel_queued_and_running(fga):
    """A queued request is dropped at once; a running one stops at its next window of steps; both report
    FGA_ERR_CANCELLED, and the server goes on serving."""
    blocker = _blocker(800)
    model = fga.model_from_medium(blocker.medium)
    server = fga.Server(model, n_workers=1)
    running = _submit(fga, server, blocker)
    queued = _submit(fga, server, blocker)
    import time
    time.sleep(0.05)                    # the first request is on the worker by now
    server.cancel(queued)
    server.cancel(running)
    for rid in (queued, running):
        with pytest.raises(fga.FGAError) as e:
            server.wait(rid)
        assert e.value.status == fga.FGA_ERR_CANCELLED
    small = W.serving_requests(n=1, seed=3, n_range=(2e3, 2e3), ks=(16.0,), np_=4, nsteps=12, dt=0.01, rx_side=4,
                               n_times=6, grid_n=32)[0].workload
    u, info = server.wait(_submit(fga, server, small))
    import torch
    assert torch.isfinite(torch.view_as_real(u)).all()
    with pytest.raises(fga.FGAError):    # a collected id is unknown
        server.cancel(running)
    server.close()


def test_device_memory_limit_gives_oom_and_recovers(fga):
    """Host-side fault injection: with a bound below what a solve needs, its allocation fails with
    FGA_ERR_OOM before cudaMalloc is called (a served request reports it as its own status while the
    server keeps serving); without the bound the same solve succeeds and the library's device memory
    returns to where it was."""
    import torch
    w = W.serving_requests(n=1, seed=3, n_range=(2e4, 2e4), ks=(16.0,), np_=4, nsteps=12, dt=0.01, rx_side=4,
                           n_times=6, grid_n=32)[0].workload
    model, desc, k = gpu_setup(w, 0)
    rx = torch.as_tensor(w.receivers, device="cuda")
    import gc
    gc.collect()                        # models and beam sets of earlier tests released first
    base = fga.device_memory_in_use()
    fga.set_device_memory_limit(base + 1e5)
    try:
        with pytest.raises(fga.FGAError) as e:
            fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
        assert e.value.status == fga.FGA_ERR_OOM
        assert fga.device_memory_in_use() == base
        server = fga.Server(model, n_workers=1)
        rid = server.submit(desc, w.dt, w.nsteps, w.times, rx, rw=w.rw, keep=k)
        with pytest.raises(fga.FGAError) as e:
            server.wait(rid)
        assert e.value.status == fga.FGA_ERR_OOM
        fga.set_device_memory_limit(0)
        u, _ = server.wait(server.submit(desc, w.dt, w.nsteps, w.times, rx, rw=w.rw, keep=k))
        assert torch.isfinite(torch.view_as_real(u)).all()
        server.close()
    finally:
        fga.set_device_memory_limit(0)
    u2, _ = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    torch.cuda.synchronize()
    assert torch.equal(u2.cpu(), u.cpu())
    gc.collect()
    assert fga.device_memory_in_use() == base
