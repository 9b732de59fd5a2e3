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
