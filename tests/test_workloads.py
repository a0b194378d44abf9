"""Host-side checks of the seeded synthetic workloads of the layered media (no GPU): the geometry the
spherical and undulating variants promise."""
import numpy as np

from paper_1810_06760_gb300 import workloads as W


def test_spherical_crust_geometry():
    w = W.shells(nq=2, np_=4, ny=16, nsteps=10, dt=0.1, n_times=2, rx_side=5, rc=60.0)
    m = w.medium
    assert m.kind == "layered" and m.layer_shape == "spheres"
    c = np.asarray(m.layer_center)
    np.testing.assert_allclose(np.linalg.norm(w.receivers - c, axis=1), 60.0, rtol=1e-12)
    np.testing.assert_allclose(m.z_interfaces, (45.0, 25.0))
    assert all(a > b for a, b in zip(m.z_interfaces, m.z_interfaces[1:]))
    # the source (10 km below the top point of the outer sphere) lies in the outer layer
    assert np.linalg.norm(np.array([0.0, 0.0, 10.0]) - c) > m.z_interfaces[0]


def test_undulating_crust_geometry():
    w = W.undulating(nq=2, np_=4, ny=16, nsteps=10, dt=0.1, n_times=2, rx_side=5)
    m = w.medium
    assert m.layer_shape == "undulating" and len(m.layer_amp) == len(m.z_interfaces) == 2
    z, a = np.asarray(m.z_interfaces), np.abs(np.asarray(m.layer_amp))
    assert np.all(np.diff(z) > a[:-1] + a[1:])              # the surfaces never touch
    assert m.layer_amp[0] * m.layer_amp[1] < 0               # opposite signs: not parallel
    assert np.all(w.receivers[:, 2] == 0.0) and np.all(z - a > 0)   # receivers above every surface
