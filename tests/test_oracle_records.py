"""Pins of the oracle's reconstruction records at sample times strictly inside an RK4 step.

The seismograms of the forward solve are sampled between step ends: inside step n at fraction
theta in (0, 1), the beam centre Q and propagation vector P are taken from the cubic Hermite
interpolant of the step's two end states and their time derivatives, and the amplitudes linearly
(the reading of the paper's sampling that the library follows; the paper itself integrates with a
fixed RK4 step and prints no sampling rule).  These tests fix that interpolation from outside:

- a homogeneous medium has straight rays, Q(t) = q + sigma c t p/|p|, constant P and amplitudes
  linear in t, so interior samples must equal the closed form at the sample time;
- in the smooth sine medium interior samples are compared with a 32x finer RK4 whose step ends fall on
  the sample times: the Hermite centre and propagation vector converge at fourth order (error ratio
  about 16 on halving dt) and the linearly interpolated amplitudes at second order (ratio about 4).

A Hermite basis with its two slope functions swapped, a missing factor dt on the slopes, theta taken
from the wrong end of the step or the amplitude weights exchanged each fail one of these.
"""
import math

import numpy as np
import pytest

from paper_1810_06760_gb300 import workloads as W


def _mesh(O, nq, qc, np_, pc, R):
    m = W.centred_mesh(nq, qc, np_, pc, R)
    return O.Mesh(m.nq, m.q0, m.dq, m.np_, m.p0, m.dp)


def _beams(O, model, cls, k=32.0):
    mesh = _mesh(O, 2, [0.45, 0.5, 0.55], 2, [0.7, -0.4, 0.5], 0.3)
    F = np.zeros((mesh.M, 3), complex)
    F[:, 0] = 1.0 + 0.2j
    F[:, 1] = 0.5j
    F[:, 2] = -0.25
    st, meta = O.beam_init(model, k, mesh, F, None, cls)
    return mesh, st, meta


def _polarised(O, rec):
    """Split records [ns, nb, 12] into Q, P and the complex polarised amplitude vector."""
    Q = rec[..., 0:3]
    P = rec[..., 3:6]
    A = rec[..., 6:12].copy().view(complex)
    return Q, P, A


@pytest.mark.parametrize("cls", [0, 1, 2, 3])
def test_interior_samples_homogeneous_closed_form(oracle, cls):
    """grad c = 0: at t = (n + theta) dt the record holds Q = q + sigma c t p/|p| and P = p to
    round-off (a cubic Hermite interpolant reproduces a straight line), and the amplitude
    a(t) = a(0)(1 - i sigma c t/(2|p|)) along P/|P| (P) or the SV/SH frame (S) up to RK4's error."""
    O = oracle
    model = O.Model("const", cp0=2.0, cs0=1.0)
    c = 2.0 if cls < 2 else 1.0
    sg = -1.0 if cls & 1 else 1.0
    mesh, st, meta = _beams(O, model, cls)
    a0 = O.state_a(st).copy()
    dt, nsteps = 0.01, 30
    times = np.array([(3 + 0.3) * dt, (11 + 0.7) * dt, (17 + 0.45) * dt, (29 + 0.9) * dt])
    s_step, s_th = O.sample_schedule(times, dt, nsteps)
    assert np.all((s_th > 0.2) & (s_th < 0.95))            # every sample is strictly inside a step
    rec = O.propagate(model, st, meta, dt, nsteps, s_step, s_th, 1.0)
    Q, P, A = _polarised(O, rec)
    q, p = mesh.points()
    pn = np.linalg.norm(p, axis=1)
    ph = p / pn[:, None]
    for j, t in enumerate(times):
        np.testing.assert_allclose(Q[j], q + sg * c * t * ph, atol=2e-14)
        np.testing.assert_allclose(P[j], p, atol=1e-15)
        fac = (1.0 - 1j * sg * c * t / (2.0 * pn))
        if cls < 2:
            want = (a0[:, 0] * fac)[:, None] * ph
        else:
            # the S frame of a straight ray is constant: N_sh = e x p/|e x p|, N_sv = N_sh x p/|p|
            e = np.where(meta[:, None] & O.META_REF_E1, [1.0, 0.0, 0.0], [0.0, 0.0, 1.0])
            nsh = np.cross(e, p)
            nsh /= np.linalg.norm(nsh, axis=1)[:, None]
            nsv = np.cross(nsh, ph)
            want = (a0[:, 0] * fac)[:, None] * nsv + (a0[:, 1] * fac)[:, None] * nsh
        np.testing.assert_allclose(A[j], want, rtol=1e-9, atol=1e-12)


def _interior_errors(O, model, cls, dt_coarse):
    """Max errors of Q, P and the polarised amplitude of interior-theta records at step dt_coarse
    against a 32x finer RK4 (dt_coarse / 32) whose step ends fall on the sample times."""
    base_dt = 0.02
    # sample times fixed in physical time: theta = 5/16 and 11/16 of a 0.02 step
    times = np.array([(n + f) * base_dt for n in (3, 8, 13) for f in (5.0 / 16.0, 11.0 / 16.0)])
    T = 16 * base_dt
    out = []
    for dt in (dt_coarse, base_dt / 32.0):
        nsteps = int(round(T / dt))
        _, st, meta = _beams(O, model, cls)
        s_step, s_th = O.sample_schedule(times, dt, nsteps)
        rec = O.propagate(model, st, meta, dt, nsteps, s_step, s_th, 1.0)
        out.append((rec, s_th))
    (rc, thc), (rf, thf) = out
    # the coarse samples are interior; the fine ones sit on step ends (theta 0 or 1 to rounding)
    assert np.all((thc > 0.2) & (thc < 0.8)), thc
    assert np.all(np.minimum(np.abs(thf), np.abs(thf - 1.0)) < 1e-9), thf
    Qc, Pc, Ac = _polarised(O, rc)
    Qf, Pf, Af = _polarised(O, rf)
    eq = np.max(np.abs(Qc - Qf))
    ep = np.max(np.abs(Pc - Pf))
    ea = np.max(np.abs(Ac - Af)) / np.max(np.abs(Af))
    return eq, ep, ea


@pytest.mark.parametrize("cls", [0, 3])
def test_interior_samples_converge_in_smooth_medium(oracle, cls):
    """Curved rays in the sine medium: Hermite Q and P at interior theta converge at order 4 (the
    interpolant and RK4 are both fourth order), the linear amplitudes at order 2."""
    O = oracle
    model = O.Model("sine", cp0=2.0, amp=0.2, cs_ratio=1.0 / math.sqrt(3.0))
    e1 = _interior_errors(O, model, cls, 0.02)
    e2 = _interior_errors(O, model, cls, 0.01)
    rq, rp, ra = e1[0] / e2[0], e1[1] / e2[1], e1[2] / e2[2]
    assert e2[0] < 1e-7 and e2[1] < 1e-6, e2
    assert 10.0 < rq < 24.0, (rq, e1, e2)
    assert 10.0 < rp < 24.0, (rp, e1, e2)
    assert 3.0 < ra < 5.5, (ra, e1, e2)
    # the amplitude error is the interpolation's, not RK4's: it dominates the Q and P errors
    assert e2[2] > 1e-7, e2
