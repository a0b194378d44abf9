"""Pins of the traveltime-misfit oracle (``oracle/traveltime.py``), none of which re-types its formulas:

* a record shifted by a whole number of samples is measured at exactly that many samples (the
  correlation is then the synthetic's autocorrelation, symmetric about the shift);
* exchanging synthetic and data negates every delay; identical records give zero delay, misfit and
  adjoint source; a shift beyond the lag range is clamped to it;
* a smooth pulse shifted by a fraction of a sample (evaluated analytically) is measured to within a
  small fraction of a sample;
* the adjoint source is the derivative of the measured delay: central finite differences of the
  oracle's own cross-correlation measurement along random smooth directions agree with
  sum Re(conj(ubar / tau) ds) when the data are a whole-sample shift of the synthetic."""
import numpy as np
import pytest

from oracle import traveltime as T


def _pulse(t, t0, width, omega, amp):
    """A complex carrier under a Gaussian envelope, per receiver and component: [n_t][n_rx][3]."""
    env = np.exp(-0.5 * ((t[:, None, None] - t0[None, :, None]) / width) ** 2)
    return amp[None] * env * np.exp(-1j * omega * (t[:, None, None] - t0[None, :, None]))


def _case(seed=0, n_t=160, n_rx=5, dt=0.005):
    rng = np.random.default_rng(seed)
    t = dt * np.arange(n_t)
    t0 = dt * rng.uniform(60, 100, n_rx)
    amp = rng.normal(size=(n_rx, 3)) + 1j * rng.normal(size=(n_rx, 3))
    return t, t0, amp, dt


def _shift(s, m):
    d = np.zeros_like(s)
    if m >= 0:
        d[m:] = s[:s.shape[0] - m]
    else:
        d[:m] = s[-m:]
    return d


@pytest.mark.parametrize("m", [-7, 0, 3, 11])
def test_whole_sample_shift_is_exact(m):
    t, t0, amp, dt = _case(1)
    s = _pulse(t, t0, 6 * dt, 60.0, amp)
    tau = T.delays(s, _shift(s, m), dt, 20)
    assert np.allclose(tau, m * dt, rtol=0, atol=1e-13)


def test_exchange_negates_and_identical_records_vanish():
    t, t0, amp, dt = _case(2)
    s = _pulse(t, t0, 6 * dt, 60.0, amp)
    rng = np.random.default_rng(5)
    d = _pulse(t, t0 + dt * rng.uniform(-4, 4, t0.size), 7 * dt, 58.0, amp * 0.8)
    a, b = T.delays(s, d, dt, 20), T.delays(d, s, dt, 20)
    assert np.allclose(a, -b, rtol=0, atol=1e-13) and np.abs(a).max() > dt
    tau, ub, mis = T.traveltime_adjoint(s, s, dt, 20)
    assert np.all(tau == 0.0) and mis == 0.0 and np.all(ub == 0.0)


def test_shift_beyond_lag_range_is_clamped():
    t, t0, amp, dt = _case(3)
    s = _pulse(t, t0, 4 * dt, 0.0, amp)
    tau = T.delays(s, _shift(s, 15), dt, 6)
    assert np.allclose(tau, 6 * dt, rtol=0, atol=1e-15)


def test_exact_tie_takes_the_smallest_lag():
    """Impulses: s at sample 50, d at samples 48 and 53 with equal weight, so C(-2) = C(3) = 1 and
    their neighbours are 0: the measurement is -2 samples (smallest lag, no sub-sample step)."""
    dt = 0.01
    s = np.zeros((100, 2, 3), complex)
    d = np.zeros_like(s)
    s[50, :, 1] = 1.0
    d[48, :, 1] = 1.0
    d[53, :, 1] = 1.0
    assert np.allclose(T.delays(s, d, dt, 10), -2 * dt, rtol=0, atol=1e-15)


@pytest.mark.parametrize("frac", [-0.4, 0.15, 0.3])
def test_sub_sample_shift_of_a_smooth_pulse(frac):
    t, t0, amp, dt = _case(4, n_rx=3)
    shift = (2 + frac) * dt
    s = _pulse(t, t0, 8 * dt, 0.0, amp)
    d = _pulse(t, t0 + shift, 8 * dt, 0.0, amp)
    tau = T.delays(s, d, dt, 10)
    assert np.abs(tau - shift).max() < 0.02 * dt


@pytest.mark.parametrize("m", [0, 4, -3])
def test_adjoint_source_is_the_derivative_of_the_measured_delay(m):
    t, t0, amp, dt = _case(6)
    s = _pulse(t, t0, 5 * dt, 70.0, amp)
    d = _shift(s, m)
    rng = np.random.default_rng(9 + m)
    tau, ub, mis = T.traveltime_adjoint(s, d, dt, 20)
    if m == 0:
        assert mis == 0.0
        tau = np.ones_like(tau)            # the direction of the delay's derivative is still defined
        ub = T.slope(s, dt) * (dt / T.norm_n(s, dt))[None, :, None]
    for _ in range(3):
        ds = _pulse(t, t0 + dt * rng.normal(size=t0.size) * 3, 7 * dt, 65.0,
                    rng.normal(size=amp.shape) + 1j * rng.normal(size=amp.shape))
        eps = 1e-7
        fd = (T.delays(s + eps * ds, d, dt, 20) - T.delays(s - eps * ds, d, dt, 20)) / (2 * eps)
        pred = np.real(np.conj(ub / tau[None, :, None]) * ds).sum(axis=(0, 2))
        assert np.allclose(fd, pred, rtol=1e-6, atol=1e-9 * dt), (fd, pred)


def test_misfit_cotangent_is_tau_times_delay_gradient():
    """d(1/2 sum tau^2) along ds equals sum Re(conj(ubar) ds) (data a whole-sample shift)."""
    t, t0, amp, dt = _case(7)
    s = _pulse(t, t0, 5 * dt, 70.0, amp)
    d = _shift(s, 5)
    _, ub, _ = T.traveltime_adjoint(s, d, dt, 20)
    rng = np.random.default_rng(3)
    ds = _pulse(t, t0 + 2 * dt, 6 * dt, 66.0, rng.normal(size=amp.shape) + 0j)
    eps = 1e-7
    mp = T.traveltime_adjoint(s + eps * ds, d, dt, 20)[2]
    mm = T.traveltime_adjoint(s - eps * ds, d, dt, 20)[2]
    fd = (mp - mm) / (2 * eps)
    pred = float(np.real(np.conj(ub) * ds).sum())
    assert abs(fd - pred) <= 1e-6 * abs(pred) + 1e-12
