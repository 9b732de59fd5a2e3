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


def _ricker_dt(t, fp, t0):
    """Time derivative of the Ricker pulse (1 - 2a) e^-a, a = (pi fp (t - t0))^2."""
    a = (np.pi * fp * (t - t0)) ** 2
    da = 2.0 * (np.pi * fp) ** 2 * (t - t0)
    return -da * np.exp(-a) * (3.0 - 2.0 * a)


def test_seismogram_chain_reproduces_the_explosion_pulse():
    """Zero contrast: every LS solve returns its background field, and the chain's traces are the
    textbook displacement of an explosion (M = I) in a homogeneous isotropic medium, radial with
    u_r(t) = [s(tau) / r^2 + s'(tau) / (alpha r)] / (4 pi rho alpha^2), tau = t - r / alpha, s the
    Ricker pulse (its near-field and far-field terms), and zero transverse motion."""
    import synthetic as sy
    med = sy.random_medium((6, 6, 6), h=20.0, seed=90, frac=0.1)
    med.dC[:] = 0.0
    med.drho[:] = 0.0
    xs = np.array([50.0, 50.0, 50.0])
    rec = np.array([[5, 0, 2], [0, 4, 5], [3, 5, 0]])
    fp, t0, df, nt, dt = 15.0, 0.1, 1.0, 500, 2e-3
    nf = 91                                   # up to 6 fp: the spectrum beyond is below 1e-15
    tr, U, its = syn.seismograms(med, nf, df, sy.explosion(), xs, rec, nt, dt, fp, t0)
    assert tr.shape == (3, 3, nt) and max(its) <= 1
    alpha = med.vp0
    t = np.arange(nt) * dt
    for r, node in enumerate(rec):
        d = node * med.h - xs
        dist = np.linalg.norm(d)
        tau = t - dist / alpha
        ur = (_ricker_time(tau, fp, t0) / dist ** 2 + _ricker_dt(tau, fp, t0) / (alpha * dist)) \
            / (4 * np.pi * med.rho0 * alpha ** 2)
        want = ur[None, :] * (d / dist)[:, None]
        assert np.abs(tr[r] - want).max() < 1e-9 * np.abs(want).max()
