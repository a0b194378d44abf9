"""The wave-packet transform (Eq. psi) and the beam amplitudes of the decomposition (Eq. alpha^k) at
the shapes the benchmark runs, through the C ABI, against the FP64 oracle's separable transform
(itself pinned equal to the direct triple sum and to the closed form of a Gaussian).

The tensor-core path (FP32: FP16 hi/lo split, FP32 accumulation in tensor memory) contracts K in
blocks of 32 complex values and tiles N at 128 complex columns, so these shapes make every stage
accumulate over several K blocks with a ragged last block (ny = 72, 100: 72 = 2x32 + 8,
100 = 3x32 + 4) and run two N tiles (A = nq np = 136, 144, 192 > 128).  The bench's own shape is
ny = 128, A = 24 x 8 = 192.

Tolerances: relative L2 per component 1e-4 (FP32 path) and 1e-10 (FP64 path), and element-wise on
the entries above 1e-3 of the largest one.  The element-wise bound follows from the arithmetic: an
FP32 sum of K <= 128 terms bounded by the peak carries an absolute error of about
sqrt(K) 2^-24 x peak per product stage (three stages), i.e. ~1e-6 of the peak, which is ~1e-3 relative
on an entry at 1e-3 of the peak; FP64: ~1e-12 of the peak, 1e-9 relative there."""
import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W
from tests.helpers import max_rel_dominant, oracle_mesh, rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 1e-10}
ELEM_TOL = {0: 3e-3, 1: 1e-8}


@pytest.fixture(scope="module")
def fga():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_06760_gb300 import build, fga as F
    build.build()
    F.lib()
    return F


def _pair_layout(F, nq, np_):
    """Oracle output in mesh order [M, 3] -> the library's per-axis pair layout [A, A, A, 3]."""
    A = nq * np_
    return (F.reshape(nq, nq, nq, np_, np_, np_, 3).transpose(0, 3, 1, 4, 2, 5, 6).reshape(A, A, A, 3))


SHAPES = [((72, 72, 72), 18, 8), ((100, 100, 100), 17, 8), ((128, 128, 128), 24, 8), ((72, 100, 128), 18, 8)]


@pytest.mark.parametrize("ny,nq,np_", SHAPES)
def test_transform_matches_oracle_at_bench_shapes(fga, oracle, ny, nq, np_):
    import torch
    f, y0, dy, mesh, k = W.transform_case(ny, nq, np_)
    ref = _pair_layout(oracle.fbi(f, y0, dy, k, oracle_mesh(oracle, mesh)), nq, np_)
    df = torch.as_tensor(f, device="cuda")
    for prec in (1, 0):
        desc = fga.init_desc(k, df, None, y0, dy, mesh, (0,), prec)
        out = fga.transform(desc).cpu().numpy()
        for c in range(3):
            e = rel_l2(out[..., c], ref[..., c])
            assert e <= TOL[prec], (prec, c, e)
        em = max_rel_dominant(out, ref)
        assert em <= ELEM_TOL[prec], (prec, em)


@pytest.mark.parametrize("prec", [1, 0])
def test_decompose_amplitudes_at_two_n_tiles(fga, oracle, prec):
    """fga_decompose end to end on a 128^3 y grid and A = 17 x 8 = 136 (two N tiles, four K blocks):
    initial amplitudes 2^{3/2} psi of P+ and S- beams (psi projected on P/|P|, resp. the SV and SH
    directions) against the oracle's initialisation from its own transform."""
    import torch
    f, y0, dy, mesh, k = W.transform_case((128, 128, 128), 17, 8)
    om = oracle.Model("sine", cp0=2.0, amp=0.2, cs_ratio=1.0 / np.sqrt(3.0))
    mdl = fga.Model("sine", cp0=2.0, amp=0.2, cs_ratio=1.0 / np.sqrt(3.0))
    omesh = oracle_mesh(oracle, mesh)
    F = oracle.fbi(f, y0, dy, k, omesh)
    df = torch.as_tensor(f, device="cuda")
    desc = fga.init_desc(k, df, None, y0, dy, mesh, (0, 3), prec)
    beams = fga.decompose(mdl, desc)
    gst, gmeta = beams.export()
    beams.close()
    n = omesh.M
    for i, cls in enumerate((0, 3)):
        ost, ometa = oracle.beam_init(om, k, omesh, F, None, cls)
        g = gst[i * n:(i + 1) * n]
        np.testing.assert_array_equal(gmeta[i * n:(i + 1) * n] & 7, ometa & 7)
        ga = g[:, 42:46].copy().view(complex)
        oa = ost[:, 42:46].copy().view(complex)
        assert rel_l2(ga, oa) <= TOL[prec], (cls, rel_l2(ga, oa))
        assert max_rel_dominant(ga, oa) <= ELEM_TOL[prec], (cls, max_rel_dominant(ga, oa))
        np.testing.assert_allclose(g[:, 0:6], ost[:, 0:6], rtol=0, atol=1e-6 if prec == 0 else 1e-14)
    mdl.close()
