"""GPU library (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 over each compared array): 1e-10 for the FP64 path, 1e-4 for the FP32
path; binning is compared bit for bit.  Beside the L2 bar, the wavefields are compared element by
element on the entries above 1e-2 of their largest one (2e-3 FP32, 1e-9 FP64): an FP32 Gaussian sum
carries an absolute error of a few 1e-6 of the peak (measured rel-L2 ~1e-5), i.e. a few 1e-4 relative
on such an entry, so a localised error in a few beams or receivers cannot hide under the L2 norm.
Sizes span several sort tiles (2048 keys), several point tiles (32 points) and ragged tails."""
import math

import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup, max_rel_dominant, oracle_beams, oracle_model, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}   # FGA_PREC_FP32, FGA_PREC_FP64
ELEM_TOL = {0: 2e-3, 1: 1e-9}
ELEM_FRAC = 1e-2


def _check_field(got, ref, prec):
    assert rel_l2(got, ref) <= TOL[prec], rel_l2(got, ref)
    em = max_rel_dominant(got, ref, ELEM_FRAC)
    assert em <= ELEM_TOL[prec], em


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _small_smooth(grid=True, **kw):
    args = dict(nq=5, np_=3, ny=24, nsteps=40, n_samples=30, rx_side=7, snap_side=5, grid_n=33, grid=grid)
    args.update(kw)
    return W.smooth(**args)


def _small_homog(**kw):
    args = dict(nq=5, np_=3, ny=20, nsteps=30, n_receivers=100)
    args.update(kw)
    return W.homogeneous(**args)


WORKLOADS = {
    "homogeneous": _small_homog,
    "sine": lambda: _small_smooth(grid=False),
    "grid": lambda: _small_smooth(grid=True),
}

GROUPS = {"Q": slice(0, 3), "P": slice(3, 6), "dzQ": slice(6, 24), "dzP": slice(24, 42), "a": slice(42, 46)}


def _compare_states(gst, gmeta, ost, ometa, tol):
    np.testing.assert_array_equal(gmeta & 7, ometa & 7)
    for name, sl in GROUPS.items():
        e = rel_l2(gst[:, sl], ost[:, sl])
        assert e <= tol, (name, e)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("wname", list(WORKLOADS))
def test_decompose_then_propagate(fga, oracle, wname, prec):
    w = WORKLOADS[wname]()
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    gst0, gmeta = beams.export()
    omodel, mesh, obeams = oracle_beams(oracle, w)
    ost0 = np.concatenate([b[1] for b in obeams])
    ometa = np.concatenate([b[2] for b in obeams])
    _compare_states(gst0, gmeta, ost0, ometa, TOL[prec])
    fga.propagate(model, beams, w.dt, w.nsteps)
    gst, gmeta = beams.export()
    ost = ost0.copy()
    oracle.propagate(omodel, ost, ometa, w.dt, w.nsteps)
    _compare_states(gst, gmeta, ost, ometa, TOL[prec])


@pytest.mark.parametrize("prec", [1, 0])
def test_reconstruct_at_points(fga, oracle, prec):
    import torch
    w = _small_smooth(grid=True, nsteps=24)
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    omodel, mesh, obeams = oracle_beams(oracle, w)
    wgt = mesh.weight(w.k)
    x = W.random_points(101, -0.1, 1.1, 4)           # 3 full tiles of 32 and a ragged one
    ref = np.zeros((x.shape[0], 3), complex)
    for cls, st, meta in obeams:
        oracle.propagate(omodel, st, meta, w.dt, w.nsteps)
        ref += oracle.gauss_sum(oracle.records(st, meta, wgt), w.k, w.rw, x)
    u = fga.reconstruct(beams, torch.as_tensor(x, device="cuda"), rw=w.rw).cpu().numpy()
    _check_field(u, ref, prec)
    # the untruncated oracle sum differs from the truncated one by at most e^-18 of the amplitudes
    ref_full = sum(oracle.gauss_sum(oracle.records(st, meta, wgt), w.k, 0.0, x) for _, st, meta in obeams)
    assert rel_l2(ref, ref_full) < 1e-6


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", ["k64", "k128", "k128_wide"])
def test_solve_seismograms_and_snapshot(fga, oracle, prec, case):
    """Whole solve against the oracle.  k = 128 (the largest wavenumber of the serving mix) makes the
    phase k P.(x - Q) reach ~68 rad inside the window, which the FP32 path reduces modulo 2 pi before
    its sine and cosine; the y grid then needs 8 ceil(sqrt(k)) = 96 points per axis."""
    import torch
    w = {"k64": lambda: _small_smooth(grid=True),
         "k128": lambda: _small_smooth(grid=True, k=128.0, ny=96),
         "k128_wide": lambda: _small_smooth(grid=True, k=128.0, ny=96, nq=6, np_=4, nsteps=60, n_samples=20)}[case]()
    model, desc, keep = gpu_setup(w, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    sn = torch.as_tensor(w.snapshot, device="cuda")
    seis, snap = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, sn, rw=w.rw)
    torch.cuda.synchronize()
    omodel = oracle_model(oracle, w.medium)
    mesh = oracle_mesh(oracle, w.mesh)
    F = oracle.fbi(w.f, w.y0, w.dy, w.k, mesh)
    ref_seis, ref_snap = oracle.solve(omodel, w.k, mesh, F, None, w.classes, w.dt, w.nsteps, w.times,
                                      w.receivers, w.rw, snap=w.snapshot)
    _check_field(seis.cpu().numpy(), ref_seis, prec)
    _check_field(snap.cpu().numpy(), ref_snap, prec)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape", [(19, 21, 1), (70, 9, 1), (9, 17, 10)])
def test_reconstruct_on_lattice(fga, oracle, prec, shape):
    """Lattice sum (per-axis factorised Gaussians) equals the oracle's brute-force sum at the same
    points; shapes give ragged tiles in every axis for both tile shapes (16x16x1 and 8x8x8)."""
    import torch
    w = _small_smooth(grid=True, nsteps=16)
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    axes = tuple(np.sort(W.random_points(1, 0, 1, 30 + a)[0, :1].tolist() + list(np.linspace(-0.05, 1.05, n)[1:]))
                 if n > 1 else np.array([0.02]) for a, n in enumerate(shape))
    axes = tuple(np.asarray(a, dtype=np.float64) for a in axes)
    u = fga.reconstruct_lattice(beams, axes, rw=w.rw).cpu().numpy()
    assert u.shape == tuple(len(a) for a in axes) + (3,)
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    omodel, mesh, obeams = oracle_beams(oracle, w)
    ref = np.zeros((X.shape[0], 3), complex)
    for cls, st, meta in obeams:
        oracle.propagate(omodel, st, meta, w.dt, w.nsteps)
        ref += oracle.gauss_sum(oracle.records(st, meta, mesh.weight(w.k)), w.k, w.rw, X)
    _check_field(u.reshape(-1, 3), ref, prec)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape", [(20, 20), (23, 45), (1, 7), (32, 20), (33, 41), (16, 16)])
def test_reconstruct_on_plane(fga, oracle, prec, shape):
    """Receiver planes (uniform axes 0 and 1, one x3): in FP32 the warp-specialised plane kernel (tiles
    of at most 32 x 20 points: one tile, several tiles with ragged edges in both axes, a single column);
    against the oracle's brute-force sum at the same points."""
    import torch
    w = _small_smooth(grid=True, nsteps=16)
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    axes = (np.linspace(0.05, 0.95, shape[0]) if shape[0] > 1 else np.array([0.41]),
            np.linspace(0.02, 0.98, shape[1]), np.array([0.3]))
    u = fga.reconstruct_lattice(beams, axes, rw=w.rw).cpu().numpy()
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    omodel, mesh, obeams = oracle_beams(oracle, w)
    ref = np.zeros((X.shape[0], 3), complex)
    for cls, st, meta in obeams:
        oracle.propagate(omodel, st, meta, w.dt, w.nsteps)
        ref += oracle.gauss_sum(oracle.records(st, meta, mesh.weight(w.k)), w.k, w.rw, X)
    _check_field(u.reshape(-1, 3), ref, prec)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("case", ["far_start_k128", "coarse_0.4", "coarse_2.0"])
def test_reconstruct_on_plane_factor_recurrence_limits(fga, oracle, prec, case):
    """Planes where the FP32 kernels' factor recurrences would leave float range: at k = 128 a 16-point
    axis whose recurrence starts 1.25 (> sqrt(174/k) = 1.17) before the beams, so the first factor
    underflows while the beams still reach the tile's far end (the runs are shortened); and planes of
    spacing 0.4 and 2.0 (k h up to 128: the ratio exp(-k h (x + h/2)) overflows unless each run is
    one point).  Against the oracle's brute-force sum."""
    import torch
    if case == "far_start_k128":
        w = _small_smooth(grid=True, nsteps=16, k=128.0, ny=96)
        axes = (np.linspace(-0.9, 0.1, 16), np.linspace(0.2, 0.7, 16), np.array([0.55]))
    elif case == "coarse_0.4":
        w = _small_smooth(grid=True, nsteps=16)
        axes = (np.linspace(-0.8, 2.0, 8), np.linspace(-1.2, 2.0, 9), np.array([0.55]))
    else:
        w = _small_smooth(grid=True, nsteps=16)
        axes = (np.linspace(-3.6, 4.4, 5), np.linspace(-1.6, 6.4, 5), np.array([0.55]))
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    u = fga.reconstruct_lattice(beams, axes, rw=w.rw).cpu().numpy().reshape(-1, 3)
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    omodel, mesh, obeams = oracle_beams(oracle, w)
    ref = np.zeros((X.shape[0], 3), complex)
    for cls, st, meta in obeams:
        oracle.propagate(omodel, st, meta, w.dt, w.nsteps)
        ref += oracle.gauss_sum(oracle.records(st, meta, mesh.weight(w.k)), w.k, w.rw, X)
    assert np.abs(ref).max() > 0 and np.isfinite(u).all()
    _check_field(u, ref, prec)


@pytest.mark.parametrize("prec", [1, 0])
def test_solve_on_lattices_equals_solve_on_points(fga, prec):
    """Receivers and snapshot given as lattices give the same seismograms and snapshot as the same
    points given one by one."""
    import torch
    w = _small_smooth(grid=True)
    model, desc, keep = gpu_setup(w, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    sn = torch.as_tensor(w.snapshot, device="cuda")
    s1, n1 = fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, sn, rw=w.rw)
    s2, n2 = fga.solve(model, desc, w.dt, w.nsteps, w.times, rw=w.rw, rx_axes=w.rx_axes, snap_axes=w.snap_axes)
    torch.cuda.synchronize()
    assert rel_l2(s2.reshape(s1.shape).cpu().numpy(), s1.cpu().numpy()) <= TOL[prec]
    assert rel_l2(n2.reshape(n1.shape).cpu().numpy(), n1.cpu().numpy()) <= TOL[prec]


@pytest.mark.parametrize("n,nc", [(0, (3, 3, 3)), (1, (2, 2, 2)), (5000, (4, 5, 6)), (20011, (9, 7, 11)),
                                  (70001, (40, 40, 40))])
def test_binning_bit_exact(fga, oracle, n, nc):
    import torch
    rng = np.random.default_rng(n + 17)
    Q = rng.uniform(-0.7, 1.8, (n, 3)).astype(np.float32)
    if n > 100:
        Q[:100] = np.float32(0.125) * rng.integers(-4, 12, (100, 3))   # exactly on cell faces
    o = np.array([-0.5, -0.25, -0.5], np.float32)
    inv_h = np.float32(1.0 / (2.25 / max(nc)))
    keys, perm, start = fga.bin_centres(torch.as_tensor(Q, device="cuda"), o, inv_h, nc)
    okey = oracle.bin_keys_f32(Q, o, inv_h, nc)
    operm, ostart = oracle.bin_sort(okey, int(np.prod(nc)))
    np.testing.assert_array_equal(keys.cpu().numpy(), okey)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    np.testing.assert_array_equal(start.cpu().numpy(), ostart)


def test_errors_are_reported_not_raised_from_device(fga):
    import torch
    w = _small_homog()
    model, desc, keep = gpu_setup(w, 1)
    desc.class_mask = 0
    with pytest.raises(fga.FGAError) as e:
        fga.decompose(model, desc)
    assert e.value.status == fga.FGA_ERR_INVALID_ARG
    desc.class_mask = 1
    beams = fga.decompose(model, desc)
    with pytest.raises(fga.FGAError):
        fga.propagate(model, beams, float("nan"), 3)
    out = fga.reconstruct(beams, torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert out.shape == (0, 3)
    with pytest.raises(fga.FGAError):   # sample time outside (0, T]
        fga.solve(model, desc, w.dt, w.nsteps, np.array([w.T * 2]), torch.as_tensor(w.receivers, device="cuda"))


@pytest.mark.parametrize("prec", [1, 0])
def test_nonfinite_input_is_reported(fga, prec):
    """Initial data holding a NaN make non-finite beams: the solve returns FGA_ERR_NUMERIC (its device
    status word) instead of silently returning NaN seismograms; the library stays usable."""
    import torch
    w = _small_smooth(grid=True, nsteps=8, n_samples=4)
    f = w.f.copy()
    f[3, 4, 5, 1] = np.nan
    model = fga.model_from_medium(w.medium, "cuda")
    df = torch.as_tensor(f, device="cuda")
    desc = fga.init_desc(w.k, df, None, w.y0, w.dy, w.mesh, w.classes, prec)
    rx = torch.as_tensor(w.receivers, device="cuda")
    with pytest.raises(fga.FGAError) as e:
        fga.solve(model, desc, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    assert e.value.status == fga.FGA_ERR_NUMERIC
    ok = torch.as_tensor(w.f, device="cuda")
    desc2 = fga.init_desc(w.k, ok, None, w.y0, w.dy, w.mesh, w.classes, prec)
    seis, _ = fga.solve(model, desc2, w.dt, w.nsteps, w.times, rx, rw=w.rw)
    assert torch.isfinite(torch.view_as_real(seis)).all()


@pytest.mark.parametrize("prec", [1, 0])
def test_export_import_resumes_propagation(fga, prec):
    """fga_beams_export, then fga_beams_import with the set's k, w and precision (fga_beams_params), then
    more steps: the same states and sums as one uninterrupted propagation (to the rounding of the Q
    compensation folded into the exported centres)."""
    import torch
    w = _small_smooth(grid=True, nsteps=24)
    model, desc, keep = gpu_setup(w, prec)
    ref = fga.decompose(model, desc)
    fga.propagate(model, ref, w.dt, 24)
    b1 = fga.decompose(model, desc)
    fga.propagate(model, b1, w.dt, 10)
    st, meta = b1.export()
    k, wt, p = fga.beams_params(b1)
    assert p == prec and k == w.k and wt > 0
    b1.close()
    b2 = fga.beams_import(st, meta, k, wt, p)
    fga.propagate(model, b2, w.dt, 14)
    s_ref, m_ref = ref.export()
    s_new, m_new = b2.export()
    np.testing.assert_array_equal(m_new, m_ref)
    tol = 1e-12 if prec == 1 else 2e-6
    for sl in (slice(0, 6), slice(6, 42), slice(42, 46)):
        assert rel_l2(s_new[:, sl], s_ref[:, sl]) <= tol, sl
    x = torch.as_tensor(W.random_points(65, 0.0, 1.0, 9), device="cuda")
    u_ref = fga.reconstruct(ref, x, rw=w.rw).cpu().numpy()
    u_new = fga.reconstruct(b2, x, rw=w.rw).cpu().numpy()
    assert rel_l2(u_new, u_ref) <= (1e-11 if prec == 1 else 1e-5)
    with pytest.raises(fga.FGAError):
        fga.beams_import(st, meta | 0x100, k, wt, p)
