"""BiCGSTAB and the relative residual of Eq. 22.  FP64, NumPy.

Test infrastructure: part of the CPU oracle (see ``oracle/__init__.py``).

The paper solves A u = u0 (Sec. 3.2) with BiCGSTAB (Van der Vorst 1992,
as in Barrett et al.'s Templates) and monitors e = ||u0 - A u|| / ||u0||
(Eq. 22).  Readings where the paper is silent: x0 = 0 unless a guess is
given, shadow residual r-hat = r0, Hermitian inner products <a, b> =
sum conj(a) b, stop on the half-step residual ||s|| as well as on ||r||,
and report the true residual of the returned iterate.
"""
from __future__ import annotations

import numpy as np

OK, BREAKDOWN, NOCONV = 0, -4, -5


def relres(apply, b, x):
    """Eq. 22: ||b - A x|| / ||b||."""
    return np.linalg.norm(b - apply(x)) / np.linalg.norm(b)


def bicgstab(apply, b, tol=1e-10, maxit=500, x0=None):
    """Solve A x = b.  Returns (x, iterations, true relative residual, status, history)."""
    b = np.asarray(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=b.dtype, copy=True)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, OK, []
    r = b - apply(x) if x0 is not None else b.copy()
    hist = [np.linalg.norm(r) / bnorm]
    if hist[-1] <= tol:
        return x, 0, relres(apply, b, x), OK, hist
    rhat = r.copy()
    rho_prev = alpha = omg = 1.0
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    status = NOCONV
    it = 0
    for it in range(1, maxit + 1):
        rho = np.vdot(rhat, r)
        if rho == 0.0 or not np.isfinite(rho):
            status = BREAKDOWN
            break
        if it == 1:
            p = r.copy()
        else:
            beta = (rho / rho_prev) * (alpha / omg)
            p = r + beta * (p - omg * v)
        v = apply(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        sn = np.linalg.norm(s) / bnorm
        if sn <= tol:
            x = x + alpha * p
            hist.append(sn)
            status = OK
            break
        t = apply(s)
        tt = np.vdot(t, t)
        omg = np.vdot(t, s) / tt
        x = x + alpha * p + omg * s
        r = s - omg * t
        rn = np.linalg.norm(r) / bnorm
        hist.append(rn)
        if rn <= tol:
            status = OK
            break
        if omg == 0.0 or not np.isfinite(omg):
            status = BREAKDOWN
            break
        rho_prev = rho
    return x, it, relres(apply, b, x), status, hist


def solve_dense(A, b):
    """Direct LU solve of the dense operator (the matrix-based method the paper replaces)."""
    shape = b.shape
    return np.linalg.solve(A, b.reshape(-1)).reshape(shape)
