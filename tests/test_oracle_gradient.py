"""Pins of the oracle's discrete adjoint: the extended-grid adjoint convolution against the dense
kernel matrix, and the full gradient of a receiver misfit against central finite differences."""
import numpy as np

import synthetic as sy
from oracle import operator as op, solver, source

W = 2 * np.pi * 12.0


def _f(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape)


def test_adjoint_convolution_equals_dense_transpose():
    med = sy.random_medium((4, 5, 3), h=9.0, seed=41)
    lam = _f(med.shape, 1)
    from oracle import green
    T = green.kernel_table(med.n, med.h, W, med.lam0, med.mu0, med.rho0)
    K = op.kernel_matrix(med.n, T)
    want = (K.conj().T @ lam.reshape(-1)).reshape(3, 5, 7, 6)
    got = op.kernel_adjoint_ext(lam, med, W)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max()


def _misfit(med, M, xs, rec, dobs, tol=1e-13):
    u0, _ = source.background_field(med.n, med.h, M, xs, W, med.lam0, med.mu0, med.rho0)
    F = op.FFTOperator(med, W)
    u, *_ = solver.bicgstab(F.apply, u0, tol=tol, maxit=500)
    d = u[:, rec[:, 2], rec[:, 1], rec[:, 0]]
    return 0.5 * np.sum(np.abs(d - dobs) ** 2), u, F


def test_gradient_matches_central_differences():
    """J = 1/2 sum |u(x_r) - d|^2: adjoint gradients w.r.t. dC (21 planes), drho and M against FD."""
    base = sy.random_medium((6, 5, 7), h=10.0, seed=42, frac=0.1)
    rng = np.random.default_rng(43)
    M = rng.standard_normal(6)
    xs = np.array([22.0, 17.0, 31.0])
    rec = np.array([[0, 0, 0], [5, 4, 6], [2, 3, 1], [4, 1, 5]])
    dobs = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    J0, u, F = _misfit(base, M, xs, rec, dobs)
    resid = u[:, rec[:, 2], rec[:, 1], rec[:, 0]] - dobs
    rhs = np.zeros_like(u)
    rhs[:, rec[:, 2], rec[:, 1], rec[:, 0]] = resid
    lam, *_ = solver.bicgstab(F.adjoint, rhs, tol=1e-13, maxit=500)
    gC, grho = op.contrast_gradient(u, lam, base, W)
    gM = source.moment_gradient(lam, base.n, base.h, xs, W, base.lam0, base.mu0, base.rho0)
    for trial in range(3):
        dC = rng.standard_normal(base.dC.shape) * 1e8
        dr = rng.standard_normal(base.drho.shape) * 20.0
        dM = rng.standard_normal(6)
        eps = 1e-3
        def J(s):
            m = sy.Medium(base.n, base.h, base.lam0, base.mu0, base.rho0, base.dC + s * dC, base.drho + s * dr)
            return _misfit(m, M + s * dM, xs, rec, dobs)[0]
        fd = (J(eps) - J(-eps)) / (2 * eps)
        an = np.sum(gC * dC) + np.sum(grho * dr) + gM @ dM
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12 * J0, (trial, fd, an)
