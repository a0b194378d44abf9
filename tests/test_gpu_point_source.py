"""The paper's accuracy experiment end to end on the GPU: the point force's radiated field at t0 = 3 s
(fga_point_force_field) is decomposed with beam selection, propagated to t1 = 6.93 s and summed on a
receiver patch of the slice y = 64 km (fga_solve), and compared with the analytic solution Eq. ex_anal
from the FP64 oracle.

The bar is the paper's own: its FGA reached 3.84% relative error against the analytic solution at
t = 6.93 s; here the relative L2 over the patch must stay below 4%.  FGA is an asymptotic method, so
this is an accuracy bar of the method, not a parity bar.  The split-precision path must agree with the
FP64 path to 1e-3 (relative L2) on the same run."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import rel_l2

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


def _run(fga, c, prec):
    import torch
    src = fga.point_force(c.x0, c.force, c.rho, c.cp, c.cs, c.f, c.T0, c.sigma)
    u, v = fga.point_force_field(src, c.ny, c.y0, c.dy, c.t0)
    model = fga.Model("const", cp0=c.cp, cs0=c.cs)
    desc = fga.init_desc(c.k, u, v, c.y0, c.dy, c.mesh, c.classes, prec, psi_rel_min=c.psi_rel_min)
    rx = torch.as_tensor(c.receivers, device="cuda")
    seis, _ = fga.solve(model, desc, c.dt, c.nsteps, [c.t1 - c.t0], rx, rw=c.rw)
    torch.cuda.synchronize()
    out = seis[0].cpu().numpy()
    model.close()
    return out


def test_point_force_fga_against_analytic_solution(fga):
    from oracle.stokes import PointForce
    c = W.e1_patch(k=0.15)
    ref = PointForce(c.x0, c.force, c.rho, c.cp, c.cs, c.f, c.T0, c.sigma).displacement(c.receivers, c.t1)
    u32 = _run(fga, c, fga.PREC_FP32)
    err = rel_l2(u32, ref)
    assert err < 0.04, err
    # the FGA sum of real data is real (the +- branches are conjugate)
    assert np.linalg.norm(u32.imag) < 1e-5 * np.linalg.norm(ref)
    u64 = _run(fga, c, fga.PREC_FP64)
    assert rel_l2(u64, ref) < 0.04
    assert rel_l2(u32, u64) < 1e-3, rel_l2(u32, u64)
