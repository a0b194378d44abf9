"""fga_reconstruct_noalloc, the Gaussian sum for callers that may not allocate device memory (for
example code in a host callback or a real-time loop that must not stall on the allocator, or a
plug-in that only receives buffers from an outside pool).  It keeps its scratch in a fixed array
inside the library instead of allocating.  Checked through the C ABI against fga_reconstruct on two
calls in a row (different point sets, so stale scratch from the first call would show), in both
precisions.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import gpu_setup, rel_l2

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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_reconstruct_twice(fga, prec):
    import torch
    w = W.smooth(nq=5, np_=3, ny=24, nsteps=20, n_samples=10, rx_side=5, snap_side=0, grid_n=33)
    model, desc, keep = gpu_setup(w, prec)
    beams = fga.decompose(model, desc)
    fga.propagate(model, beams, w.dt, w.nsteps)
    cdt = torch.complex64 if prec == 0 else torch.complex128
    # the warm-up call (no points) does only the one-time lookup of the scratch array
    fga.reconstruct_noalloc(beams, torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                            torch.empty((0, 3), dtype=cdt, device="cuda"), rw=w.rw)
    for n, seed in ((101, 1), (57, 2)):
        x = torch.as_tensor(W.random_points(n, -0.1, 1.1, seed), device="cuda")
        ref = fga.reconstruct(beams, x, rw=w.rw)
        out = torch.full((n, 3), float("nan"), dtype=cdt, device="cuda")
        fga.reconstruct_noalloc(beams, x, out, rw=w.rw)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= TOL[prec]


def test_noalloc_rejects_too_many_points(fga):
    import torch
    w = W.homogeneous(nq=3, np_=2, ny=12, nsteps=2)
    model, desc, keep = gpu_setup(w, 0)
    beams = fga.decompose(model, desc)
    x = torch.zeros((4097, 3), dtype=torch.float64, device="cuda")
    out = torch.empty((4097, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(fga.FGAError) as e:
        fga.reconstruct_noalloc(beams, x, out)
    assert e.value.status == fga.FGA_ERR_INVALID_ARG and "4096" in str(e.value)
