"""Time-domain receiver traces from frequency-domain solutions (Sec. 4.1.2).  FP64, NumPy.

Test infrastructure: part of the CPU oracle (see ``oracle/__init__.py``).

The paper solves at positive and negative frequencies up to Nyquist and inverse-Fourier
transforms the receiver data.  With time dependence exp(-i w t) and a real medium, U(-f) =
conj(U(f)), so for equally spaced frequencies f_k = k df (k = 0..K):

    u(t) = df * [ W_0 U_0 + 2 Re sum_{k>=1} W_k U_k exp(-2 pi i f_k t) ],

W the source wavelet's spectrum.  Wavelet: Ricker with peak frequency fp delayed by t0,
W(f) = 2 f^2 / (sqrt(pi) fp^3) exp(-f^2 / fp^2) exp(+2 pi i f t0) (Tables 1 and 3 use fp = 60 Hz).
"""
from __future__ import annotations

import numpy as np


def ricker_spectrum(f, fp, t0):
    f = np.asarray(f, dtype=np.float64)
    return 2.0 * f * f / (np.sqrt(np.pi) * fp ** 3) * np.exp(-(f / fp) ** 2) * np.exp(2j * np.pi * f * t0)


def traces(spectra, df, nt, dt, fp, t0):
    """spectra (K+1, ...) complex at f_k = k df, k = 0..K -> real traces (..., nt) at t = j dt."""
    spectra = np.asarray(spectra)
    K1 = spectra.shape[0]
    f = np.arange(K1) * df
    W = ricker_spectrum(f, fp, t0)
    t = np.arange(nt) * dt
    ph = np.exp(-2j * np.pi * f[:, None] * t[None, :])          # (K+1, nt)
    wgt = np.full(K1, 2.0)
    wgt[0] = 1.0
    S = (wgt * W)[:, None] * ph                                 # (K+1, nt)
    out = np.tensordot(spectra, S, axes=([0], [0]))            # (..., nt) complex
    return df * np.real(out)


def seismograms(medium, nf, df, M, xs, receivers, nt, dt, fp, t0, mode="exact", tol=1e-12, maxit=1000):
    """The whole chain of Sec. 4.1.2 for one moment-tensor source: for f_k = k df, k = 1 .. nf-1,
    solve the LS system A_k u_k = u0_k (Eqs. 13-16, 21, 22) with the oracle's BiCGSTAB, read the
    three displacement components at the receiver nodes, and synthesise the traces above.  The
    k = 0 row stays zero (the Ricker weight W_0 is zero).

    receivers: (nrec, 3) integer node indices (ix, iy, iz).  Returns (traces (nrec, 3, nt),
    spectra (nf, nrec, 3), iterations per frequency)."""
    from . import operator as _op, solver as _solver, source as _source
    rec = np.asarray(receivers, dtype=int)
    U = np.zeros((nf, rec.shape[0], 3), dtype=np.complex128)
    iters = [0] * nf
    for k in range(1, nf):
        w = 2.0 * np.pi * k * df
        F = _op.FFTOperator(medium, w, mode)
        u0, _ = _source.background_field(medium.n, medium.h, M, xs, w, medium.lam0, medium.mu0, medium.rho0, mode)
        u, it, _, status, _ = _solver.bicgstab(F.apply, u0, tol=tol, maxit=maxit)
        if status != _solver.OK:
            raise RuntimeError(f"oracle solve at {k * df} Hz did not converge")
        iters[k] = it
        for r, (ix, iy, iz) in enumerate(rec):
            U[k, r, :] = u[:, iz, iy, ix]
    return traces(U, df, nt, dt, fp, t0), U, iters
