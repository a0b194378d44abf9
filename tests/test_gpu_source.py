"""The point-force field (Eq. ex_anal and its time derivative) through the C ABI against the FP64
oracle's closed form (complex error function, itself pinned by the wave equation, Kelvin's static
solution and quadrature).  The library integrates the near-field term by composite Gauss-Legendre
quadrature, so agreement to ~1e-12 of the field's scale checks both independently."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-11


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _grid_points(ny, y0, dy):
    ax = [y0[a] + dy[a] * np.arange(ny[a]) for a in range(3)]
    return np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)


def _src(fga, S):
    return fga.point_force(S.x0, S.d, S.rho, S.cp, S.cs, S.f, S.T0, S.sigma)


@pytest.mark.parametrize("t", [0.0, 3.0, 6.93])
def test_point_force_field_matches_oracle(fga, t):
    from oracle.stokes import e1_source
    S = e1_source(d=(1.0, 1.0, 1.0))
    # a ragged grid through the source point itself, out to ~60 km
    ny, dy = (23, 17, 11), (5.3, 4.1, 7.7)
    y0 = (64.0 - 11 * 5.3, 64.0 - 8 * 4.1, 64.0 - 5 * 7.7)
    u, v = fga.point_force_field(_src(fga, S), ny, y0, dy, t)
    x = _grid_points(ny, y0, dy)
    uo = S.displacement(x, t)
    vo = S.velocity(x, t)
    ug = u.cpu().numpy().reshape(-1, 3)
    vg = v.cpu().numpy().reshape(-1, 3)
    assert np.all(ug.imag == 0) and np.all(vg.imag == 0)
    src = np.nonzero(np.all(np.abs(x - S.x0) < 1e-9, axis=1))[0]
    assert src.size == 1 and np.all(ug[src] == 0) and np.all(vg[src] == 0)
    for got, want in ((ug.real, uo), (vg.real, vo)):
        scale = np.abs(want).max()
        assert scale > 0
        np.testing.assert_allclose(got, want, rtol=0, atol=TOL * scale)


def test_point_force_static_limit_and_options(fga):
    """f = 0 and a very long pulse (the oracle's Kelvin limit); only the displacement requested.  With
    sigma = 1000 s the oracle's closed form subtracts sigma^2/2 (g(w2) - g(w1)) from terms of size
    sigma^2, which leaves it ~1e-9 relative, so the bar here is 1e-8."""
    from oracle.stokes import PointForce
    S = PointForce(np.array([1.0, 2.0, 3.0]), np.array([0.3, -0.5, 0.8]), 2.5, 6.0, 3.5, 0.0, 0.0, 1000.0)
    ny, y0, dy = (9, 8, 7), (-3.0, -2.0, -1.0), (1.1, 1.3, 1.7)
    u, _ = fga.point_force_field(_src(fga, S), ny, y0, dy, 3.0, velocity=False)
    x = _grid_points(ny, y0, dy)
    want = S.displacement(x, 3.0)
    np.testing.assert_allclose(u.cpu().numpy().reshape(-1, 3).real, want, rtol=0, atol=1e-8 * np.abs(want).max())


def test_point_force_rejections(fga):
    from oracle.stokes import e1_source
    S = e1_source()
    for bad in ({"cs": 9.0}, {"rho": 0.0}, {"sigma": -1.0}, {"f": -1.0}):
        kw = {"x0": S.x0, "force": S.d, "rho": S.rho, "cp": S.cp, "cs": S.cs, "f": S.f, "T0": S.T0,
              "sigma": S.sigma}
        kw.update(bad)
        with pytest.raises(fga.FGAError):
            fga.point_force_field(fga.point_force(**kw), (4, 4, 4), (0, 0, 0), (1, 1, 1), 1.0)
    with pytest.raises(fga.FGAError):
        fga.point_force_field(_src(fga, S), (4, 0, 4), (0, 0, 0), (1, 1, 1), 1.0)
