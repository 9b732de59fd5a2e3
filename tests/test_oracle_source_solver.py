"""Pins of the oracle's moment-tensor source (Eqs. 13-16) and BiCGSTAB (Sec. 3.2, Eq. 22)."""
import numpy as np
import pytest

import synthetic as sy
from oracle import green, operator as op, source, solver

LAM, MU = sy.iso_lame(3000.0, 1730.0, 2300.0)
RHO = 2300.0


def test_explosion_far_field_is_outward_p_pulse():
    """M = I: u0 -> -i k_alpha g exp(i k r) / (4 pi rho alpha^2 r) radially (outward for a positive moment rate)."""
    w = 2 * np.pi * 30.0
    alpha = 3000.0
    d = np.array([0.2, 0.6, -0.7])
    d /= np.linalg.norm(d)
    for r in (2000.0, 20000.0):
        xs = np.array([0.0, 0.0, 0.0])
        # evaluate on a 1-node "grid" placed at d*r by shifting the source instead
        u0, hit = source.background_field((1, 1, 1), 1.0, sy.explosion(), -d * r, w, LAM, MU, RHO)
        assert not hit
        k = w / alpha
        far = -1j * k * d * np.exp(1j * k * r) / (4 * np.pi * RHO * alpha ** 2 * r)
        err = np.abs(u0[:, 0, 0, 0] - far).max() / np.abs(far).max()
        assert err < 3.0 / (k * r)
        del xs


def test_source_linear_in_moment_and_matches_dgreen():
    n = (4, 3, 5)
    h = 10.0
    w = 2 * np.pi * 10
    xs = np.array([13.0, 7.0, 22.0])
    rng = np.random.default_rng(0)
    M1, M2 = rng.standard_normal(6), rng.standard_normal(6)
    u1, _ = source.background_field(n, h, M1, xs, w, LAM, MU, RHO)
    u2, _ = source.background_field(n, h, M2, xs, w, LAM, MU, RHO)
    u12, _ = source.background_field(n, h, 2 * M1 - 3 * M2, xs, w, LAM, MU, RHO)
    assert np.allclose(u12, 2 * u1 - 3 * u2, rtol=1e-13, atol=1e-30)
    # one node by hand: u0_i = -sum_jk M_jk dG_ij/dx_k (x - s), M12 = M21 picked from Voigt slot 6
    x = np.array([2 * h, 1 * h, 3 * h])
    dG = green.dgreen((x - xs)[None, :], w, LAM, MU, RHO)[0]
    M = source.moment_3x3(M1)
    assert M[0, 1] == M1[5] and M[1, 2] == M1[3] and M[0, 2] == M1[4]
    want = -np.einsum("ijk,jk->i", dG, M)
    assert np.allclose(u1[:, 3, 1, 2], want, rtol=1e-13)


def test_source_derivative_by_richardson_on_source_position():
    """u0_i(x) = M_jk dG_ij(x - xi)/d xi_k at xi = s: differentiate the oracle's G numerically in s."""
    w = 2 * np.pi * 12
    x = np.array([[30.0, -20.0, 10.0]])
    s = np.array([1.0, 2.0, -3.0])
    rng = np.random.default_rng(1)
    M6 = rng.standard_normal(6)
    M = source.moment_3x3(M6)
    num = np.zeros(3, dtype=complex)
    for k in range(3):
        def fd(step):
            e = np.zeros(3)
            e[k] = step
            return (green.green(x - (s + e), w, LAM, MU, RHO) - green.green(x - (s - e), w, LAM, MU, RHO))[0] / (2 * step)
        dGk = (4 * fd(1e-3) - fd(2e-3)) / 3                 # d G(x - xi) / d xi_k
        num += np.einsum("ij,j->i", dGk, M[:, k])
    u0, _ = source.background_field((1, 1, 1), 1.0, M6, s - x[0], w, LAM, MU, RHO)
    assert np.abs(u0[:, 0, 0, 0] - num).max() / np.abs(num).max() < 1e-9


def test_source_on_node_is_zero_and_flagged():
    u0, hit = source.background_field((3, 3, 3), 10.0, sy.explosion(), np.array([10.0, 10.0, 10.0]),
                                      2 * np.pi * 5, LAM, MU, RHO)
    assert hit
    assert np.all(u0[:, 1, 1, 1] == 0)
    assert np.all(np.abs(u0[:, 0, 0, 0]) > 0)


def test_bicgstab_matches_dense_lu():
    med = sy.random_medium((5, 4, 6), seed=11, frac=0.15)
    w = 2 * np.pi * 15
    u0, _ = source.background_field(med.n, med.h, sy.double_couple_12(), np.array([17.0, 13.0, 21.0]),
                                    w, med.lam0, med.mu0, med.rho0)
    A = op.dense_matrix(med, w)
    xd = solver.solve_dense(A, u0)
    F = op.FFTOperator(med, w)
    x, it, rr, st, hist = solver.bicgstab(F.apply, u0, tol=1e-12, maxit=300)
    assert st == solver.OK
    assert rr <= 1e-11
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10
    # Eq. 22 residual of the dense solution is at rounding level
    assert solver.relres(F.apply, u0, xd) < 1e-13


def test_bicgstab_trivial_cases():
    med = sy.random_medium(3, seed=12)
    F = op.FFTOperator(med, 2 * np.pi * 5)
    z = np.zeros((3, 3, 3, 3), dtype=complex)
    x, it, rr, st, _ = solver.bicgstab(F.apply, z)
    assert it == 0 and np.all(x == 0) and st == solver.OK
    med.dC[:] = 0
    med.drho[:] = 0
    F = op.FFTOperator(med, 2 * np.pi * 5)
    b = np.ones((3, 3, 3, 3), dtype=complex)
    x, it, rr, st, _ = solver.bicgstab(F.apply, b, tol=1e-12)
    # A = I: one iteration, half step exits with s = 0
    assert it == 1 and np.allclose(x, b) and rr == 0.0


def test_bicgstab_converges_on_inclusion_workload():
    """16^3 VTI cube inclusion, explosion at the centre, 10 Hz: a few iterations to 1e-10 (Sec. 4.1.1)."""
    wl = sy.get_workload("inclusion16_fp64")
    med = wl.medium()
    M, xs = wl.sources()
    w = 2 * np.pi * wl.freqs_hz[0]
    u0, hit = source.background_field(med.n, med.h, M[0], xs[0], w, med.lam0, med.mu0, med.rho0)
    assert not hit
    F = op.FFTOperator(med, w)
    x, it, rr, st, hist = solver.bicgstab(F.apply, u0, tol=1e-10, maxit=100)
    assert st == solver.OK and rr < 1e-9
    assert it <= 12
