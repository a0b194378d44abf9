"""fga_traveltime_adjoint (CUDA) against the FP64 oracle (oracle/traveltime.py) on the same seeded records:
delays, adjoint source and misfit element by element, in both record precisions, with lag ranges
narrower and wider than one CTA's threads, ties, identical records, a one-sample record, no receivers,
a zero lag range and argument errors; then on FGA seismograms of the crosswell geometry (background
against perturbed model), the records the traveltime gradient is taken on."""
import numpy as np
import pytest

from oracle import traveltime as T
from paper_1810_06760_gb300 import workloads as W

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


def _records(seed, n_t, n_rx, dt, max_shift):
    rng = np.random.default_rng(seed)
    t = dt * np.arange(n_t)
    t0 = dt * rng.uniform(0.35 * n_t, 0.65 * n_t, n_rx)
    w = dt * rng.uniform(3, 9, n_rx)
    om = rng.uniform(0.0, 1.2 / dt, n_rx)
    amp = rng.normal(size=(n_rx, 3)) + 1j * rng.normal(size=(n_rx, 3))
    sh = dt * rng.uniform(-max_shift, max_shift, n_rx)
    sh[:3] = dt * np.round(sh[:3] / dt)                       # some whole-sample shifts

    def pulse(tc, scale):
        x = (t[:, None] - tc[None, :]) / w[None, :]
        return (np.exp(-0.5 * x * x) * np.exp(-1j * om[None, :] * (t[:, None] - tc[None, :])))[:, :, None] * amp[None] * scale

    s = pulse(t0, 1.0)
    d = pulse(t0 + sh, 0.9) + 0.02 * (rng.normal(size=s.shape) + 1j * rng.normal(size=s.shape))
    return s, d


def _run(fga, s, d, dt, M, cdt):
    import torch
    ts = torch.as_tensor(s.astype(cdt), device="cuda")
    td = torch.as_tensor(d.astype(cdt), device="cuda")
    tau, ub, mis = fga.traveltime_adjoint(ts, td, dt, M)
    torch.cuda.synchronize()
    return tau.cpu().numpy(), ub.cpu().numpy(), float(mis.cpu()[0])


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n_t,n_rx,M", [(300, 37, 40), (700, 9, 300), (64, 3, 63)])
@pytest.mark.parametrize("cdt", [np.complex128, np.complex64])
def test_parity_with_oracle(fga, n_t, n_rx, M, cdt):
    dt = 0.004
    s, d = _records(n_t + n_rx, n_t, n_rx, dt, 0.8 * M + 2)
    s, d = s.astype(cdt), d.astype(cdt)                       # the oracle sees the same stored values
    tau, ub, mis = _run(fga, s, d, dt, M, cdt)
    otau, oub, omis = T.traveltime_adjoint(s, d, dt, M)
    assert np.abs(tau - otau).max() <= 1e-12 * max(np.abs(otau).max(), dt)
    assert abs(mis - omis) <= 1e-12 * max(omis, 1e-30)
    assert _rel(ub, oub) <= (1e-12 if cdt == np.complex128 else 2e-7)
    assert np.abs(otau).max() > 2 * dt                          # the case exercises real shifts


def test_edge_cases(fga):
    import torch
    dt = 0.01
    # identical records, exact tie (impulses), a one-sample record, a zero lag range
    s = np.zeros((100, 4, 3), np.complex128)
    d = np.zeros_like(s)
    s[50, :, 1] = 1.0
    d[48, :, 1] = 1.0
    d[53, :, 1] = 1.0
    s[:, 3] = d[:, 3]                                           # receiver 3: identical records
    for M in (10, 0):
        tau, ub, mis = _run(fga, s, d, dt, M, np.complex128)
        otau, oub, omis = T.traveltime_adjoint(s, d, dt, M)
        assert np.array_equal(tau, otau) and abs(mis - omis) <= 1e-15
        assert _rel(ub, oub) <= 1e-13 or np.abs(oub).max() == 0
    assert np.allclose(_run(fga, s, d, dt, 10, np.complex128)[0][:3], -2 * dt, atol=1e-15)
    one = np.ones((1, 2, 3), np.complex128)
    tau, ub, mis = _run(fga, one, one, dt, 0, np.complex128)
    assert np.all(tau == 0) and mis == 0 and np.all(ub == 0)
    empty = torch.zeros((5, 0, 3), dtype=torch.complex64, device="cuda")
    tau, ub, mis = fga.traveltime_adjoint(empty, empty, dt, 2)
    assert tau.numel() == 0 and float(mis.cpu()[0]) == 0.0


def test_argument_errors(fga):
    import torch
    x = torch.zeros((10, 2, 3), dtype=torch.complex64, device="cuda")
    for dt, M in ((0.01, 10), (0.01, -1), (0.0, 2), (float("nan"), 2)):
        with pytest.raises(fga.FGAError) as e:
            fga.traveltime_adjoint(x, x, dt, M)
        assert e.value.status == 1 and "fga_traveltime_adjoint" in str(e.value)
    long = torch.zeros((3000, 1, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(fga.FGAError) as e:
        fga.traveltime_adjoint(long, long, 0.01, 5)
    assert "shared-memory" in str(e.value)


@pytest.mark.parametrize("prec", [0, 1])
def test_parity_on_crosswell_seismograms(fga, prec):
    """Records of a small crosswell case: synthetic on the background model, data on the perturbed one."""
    import torch
    ws, true = W.crosswell(n_src_side=1, nq=4, np_=4, ny=32, nsteps=40, grid_n=17, rx_side=4, n_times=40)
    w = ws[0]
    cdt = torch.complex64 if prec == 0 else torch.complex128
    f = torch.as_tensor(w.f, device="cuda")
    desc = fga.init_desc(w.k, f, None, w.y0, w.dy, w.mesh, w.classes, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    s, _ = fga.solve(fga.model_from_medium(w.medium), desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    d, _ = fga.solve(fga.model_from_medium(true), desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    dt = float(w.times[1] - w.times[0])
    assert np.allclose(np.diff(w.times), dt)
    tau, ub, mis = fga.traveltime_adjoint(s.to(cdt), d.to(cdt), dt, 10)
    torch.cuda.synchronize()
    otau, oub, omis = T.traveltime_adjoint(s.cpu().numpy(), d.cpu().numpy(), dt, 10)
    tau, ub = tau.cpu().numpy(), ub.cpu().numpy()
    assert np.abs(tau - otau).max() <= 1e-12 * max(np.abs(otau).max(), dt)
    assert _rel(ub, oub) <= (1e-12 if prec == 1 else 2e-7)
    assert abs(float(mis.cpu()[0]) - omis) <= 1e-12 * max(omis, 1e-30)


def test_autograd_traveltime_misfit(fga):
    """adjoint.traveltime_misfit: value = the oracle's misfit; u.grad = the oracle's adjoint source (torch keeps
    dL/dRe u + i dL/dIm u for a real loss); a scaled loss scales the gradient."""
    import torch
    from paper_1810_06760_gb300 import adjoint as A
    dt = 0.004
    s, d = _records(11, 200, 6, dt, 12)
    for cdt, tol in ((torch.complex128, 1e-12), (torch.complex64, 2e-7)):
        u = torch.as_tensor(s, device="cuda").to(cdt).requires_grad_(True)
        dd = torch.as_tensor(d, device="cuda").to(cdt)
        L = 3.0 * A.traveltime_misfit(u, dd, dt, 16)
        L.backward()
        _, oub, omis = T.traveltime_adjoint(u.detach().cpu().numpy(), dd.cpu().numpy(), dt, 16)
        assert abs(float(L.detach()) - 3.0 * omis) <= 1e-12 * 3.0 * omis
        assert _rel(u.grad.cpu().numpy(), 3.0 * oub) <= tol
