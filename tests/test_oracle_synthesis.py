"""Pins of the oracle's time-domain synthesis: a flat spectrum returns the Ricker pulse in closed form,
a pure delay shifts it, and linearity."""
import numpy as np

from oracle import synthesis as syn


def _ricker_time(t, fp, t0):
    a = (np.pi * fp * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def test_flat_spectrum_gives_ricker_pulse():
    fp, t0, dt, nt = 60.0, 0.05, 3e-4, 800
    df = 1.0 / (nt * dt) / 4.0            # fine frequency sampling: the periodic images are far away
    K = int(600.0 / df)                    # the Ricker spectrum is negligible beyond 10 fp
    tr = syn.traces(np.ones(K + 1), df, nt, dt, fp, t0)
    want = _ricker_time(np.arange(nt) * dt, fp, t0)
    assert np.abs(tr - want).max() < 1e-6


def test_delay_and_linearity():
    fp, t0, dt, nt = 40.0, 0.06, 5e-4, 500
    df = 0.25
    f = np.arange(int(500 / df) + 1) * df
    tau = 0.02
    tr = syn.traces(np.exp(2j * np.pi * f * tau), df, nt, dt, fp, t0)      # delay by tau
    want = _ricker_time(np.arange(nt) * dt, fp, t0 + tau)
    assert np.abs(tr - want).max() < 1e-6
    rng = np.random.default_rng(0)
    A = rng.standard_normal((f.size, 2)) + 1j * rng.standard_normal((f.size, 2))
    B = rng.standard_normal((f.size, 2)) + 1j * rng.standard_normal((f.size, 2))
    lhs = syn.traces(2 * A - B, df, 50, dt, fp, t0)
    assert np.allclose(lhs, 2 * syn.traces(A, df, 50, dt, fp, t0) - syn.traces(B, df, 50, dt, fp, t0))
