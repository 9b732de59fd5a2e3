"""Pins of the oracle's discrete LS operator (Eqs. 8, 11, 17-21).

Independent routes: the dense matrix (direct sums, sparse Kronecker
difference operators) against the FFT form of Eq. 21 (spectral i kappa
factors); closed forms for single-voxel scatterers; exactness of the
finite-difference strain on polynomials; the PDE of Eq. 1 by finite
differences for the sign of every term.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle import green, operator as op, source, solver

W10 = 2 * np.pi * 10.0


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape)


def test_strain_exact_on_linear_field():
    """u = B x (any B): every node, boundaries included, gets the exact engineering strain."""
    n = (5, 4, 6)
    h = 3.0
    rng = np.random.default_rng(1)
    B = rng.standard_normal((3, 3))
    Z, Y, X = np.meshgrid(np.arange(6) * h, np.arange(4) * h, np.arange(5) * h, indexing="ij")
    xyz = np.stack([X, Y, Z])
    u = np.einsum("ij,j...->i...", B, xyz)
    e = op.strain(u, h)
    want = [B[0, 0], B[1, 1], B[2, 2], B[1, 2] + B[2, 1], B[0, 2] + B[2, 0], B[0, 1] + B[1, 0]]
    for J in range(6):
        assert np.allclose(e[J], want[J], rtol=1e-12, atol=1e-12)
    assert e.shape == (6, 6, 4, 5)
    del n


def test_strain_quadratic_interior_central_boundary_one_sided():
    h = 2.0
    x = np.arange(7) * h
    f = x ** 2
    d = op._d_axis(f, 0, h)
    assert np.allclose(d[1:-1], 2 * x[1:-1])              # central difference exact on quadratics
    assert d[0] == pytest.approx((f[1] - f[0]) / h)       # first-order one-sided at the ends
    assert d[-1] == pytest.approx((f[-1] - f[-2]) / h)


def test_stress_isotropic_contrast():
    """An isotropic contrast (dlam, dmu) gives sigma = dlam tr(eps) I + dmu * engineering shear."""
    dlam, dmu = 3.0, 5.0
    C = sy.iso_voigt(dlam, dmu)
    dC21 = sy.pack21(C)[:, None]
    rng = np.random.default_rng(2)
    eps = rng.standard_normal((6, 1))
    s = op.stress(dC21, eps)
    tr = eps[0] + eps[1] + eps[2]
    assert np.allclose(s[:3], dlam * tr + 2 * dmu * eps[:3])
    assert np.allclose(s[3:], dmu * eps[3:])


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_dense_equals_fft(mode):
    """Eq. 21 (FFT, i kappa factors) reproduces the direct-sum operator to rounding, non-cubic grid."""
    med = sy.random_medium((4, 5, 3), h=10.0, seed=1)
    u = _field(med.shape, 3)
    A = op.dense_matrix(med, W10, mode)
    Ad = (A @ u.reshape(-1)).reshape(u.shape)
    Af = op.FFTOperator(med, W10, mode).apply(u)
    assert np.linalg.norm(Ad - Af) / np.linalg.norm(Ad) < 1e-13
    # and the scattered part is not negligible (the test has teeth)
    assert np.linalg.norm(u - Af) / np.linalg.norm(u) > 1e-2


def test_direct_sum_equals_fft():
    med = sy.random_medium((3, 4, 4), h=8.0, seed=2)
    u = _field(med.shape, 4)
    a = op.apply_direct(u, med, W10)
    b = op.FFTOperator(med, W10).apply(u)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13
    # the multi-threaded transform (scipy.fft, used to time the oracle on all cores) is the same
    # operator: it matches the direct sums too
    c = op.FFTOperator(med, W10, workers=2).apply(u)
    assert np.linalg.norm(a - c) / np.linalg.norm(a) < 1e-13


def test_zero_contrast_is_identity():
    med = sy.random_medium(4, seed=3)
    med.dC[:] = 0.0
    med.drho[:] = 0.0
    u = _field(med.shape, 5)
    assert np.array_equal(op.FFTOperator(med, W10).apply(u), u) or \
        np.abs(op.FFTOperator(med, W10).apply(u) - u).max() == 0.0


def test_single_voxel_density_scatterer_closed_form():
    """Only drho at node a: K u = w^2 drho T(x - a) u(a), and the full solve is closed form."""
    n = (5, 5, 5)
    h = 10.0
    lam, mu = sy.iso_lame(3000.0, 1730.0, 2300.0)
    dC = np.zeros((21, 5, 5, 5))
    drho = np.zeros((5, 5, 5))
    a = (2, 1, 3)  # (x, y, z)
    drho[a[2], a[1], a[0]] = 400.0
    med = sy.Medium(n, h, lam, mu, 2300.0, dC, drho)
    T = green.kernel_table(n, h, W10, lam, mu, 2300.0)
    col = lambda c: source.point_force_field(n, h, T, a, c)  # noqa: E731  T(x - a) e_c
    u = _field((5, 5, 5), 6)
    F = op.FFTOperator(med, W10)
    Ku = u - F.apply(u)
    ua = u[:, a[2], a[1], a[0]]
    want = W10 ** 2 * 400.0 * sum(col(c) * ua[c] for c in range(3))
    assert np.abs(Ku - want).max() / np.abs(want).max() < 1e-13
    # full solution: u(a) = (I - w^2 drho T(0))^{-1} u0(a), u = u0 + w^2 drho T(x - a) u(a)
    u0 = _field((5, 5, 5), 7)
    T0 = T[:, :, 0, 0, 0]
    ua = np.linalg.solve(np.eye(3) - W10 ** 2 * 400.0 * T0, u0[:, a[2], a[1], a[0]])
    usol = u0 + W10 ** 2 * 400.0 * sum(col(c) * ua[c] for c in range(3))
    x, it, rr, st, _ = solver.bicgstab(F.apply, u0, tol=1e-13, maxit=50)
    assert st == 0
    assert np.linalg.norm(x - usol) / np.linalg.norm(usol) < 1e-11


def test_single_voxel_stiffness_scatterer_stencil():
    """Only dC at node a: u_s(x) = sum_k [T(x - a + e_k) - T(x - a - e_k)] sigma_.k(a) / 2h.

    sigma(a) = dC eps(a), eps from the central differences of u around a.
    """
    n = (6, 5, 7)
    h = 10.0
    lam, mu = sy.iso_lame(3000.0, 1730.0, 2300.0)
    rng = np.random.default_rng(8)
    a = (2, 3, 4)
    C6 = rng.standard_normal((6, 6)) * 1e9
    C6 = C6 + C6.T
    dC = np.zeros((21, 7, 5, 6))
    dC[:, a[2], a[1], a[0]] = sy.pack21(C6)
    med = sy.Medium(n, h, lam, mu, 2300.0, dC, np.zeros((7, 5, 6)))
    T = green.kernel_table(n, h, W10, lam, mu, 2300.0)
    u = _field((7, 5, 6), 9)

    def at(c, dx=0, dy=0, dz=0):
        return u[c, a[2] + dz, a[1] + dy, a[0] + dx]

    def du(c, k):  # central difference of u_c along axis k at a
        e = [0, 0, 0]
        e[k] = 1
        return (at(c, *e) - at(c, *[-v for v in e])) / (2 * h)

    eps = np.array([du(0, 0), du(1, 1), du(2, 2), du(1, 2) + du(2, 1), du(0, 2) + du(2, 0), du(0, 1) + du(1, 0)])
    sig6 = C6 @ eps
    S = np.array([[sig6[0], sig6[5], sig6[4]], [sig6[5], sig6[1], sig6[3]], [sig6[4], sig6[3], sig6[2]]])
    want = np.zeros((3, 7, 5, 6), dtype=complex)
    for k in range(3):
        e = [0, 0, 0]
        e[k] = 1
        plus = tuple(a[i] - e[i] for i in range(3))    # T(x - (a - e_k)) = T(x - a + e_k)
        minus = tuple(a[i] + e[i] for i in range(3))
        for j in range(3):
            want += (source.point_force_field(n, h, T, plus, j)
                     - source.point_force_field(n, h, T, minus, j)) * S[j, k] / (2 * h)
    got = u - op.FFTOperator(med, W10).apply(u)
    assert np.abs(got - want).max() / np.abs(want).max() < 1e-12


def test_adjoint_dot_product_and_dense():
    med = sy.random_medium((4, 3, 5), seed=4)
    F = op.FFTOperator(med, W10)
    v = _field(med.shape, 10)
    w = _field(med.shape, 11)
    lhs = np.vdot(w, F.apply(v))
    rhs = np.vdot(F.adjoint(w), v)
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    A = op.dense_matrix(med, W10)
    AH = (A.conj().T @ w.reshape(-1)).reshape(w.shape)
    assert np.linalg.norm(F.adjoint(w) - AH) / np.linalg.norm(AH) < 1e-13


def test_born_linearity():
    """u(eps dC) - u0 - eps K u0 = O(eps^2): the log-log slope is 2."""
    base = sy.random_medium(6, seed=5, frac=0.2)
    x0 = np.array([2.5, 2.5, 2.5]) * base.h
    u0, _ = source.background_field(base.n, base.h, sy.explosion(), x0, W10, base.lam0, base.mu0, base.rho0)
    errs = []
    epss = [1e-2, 1e-3]
    for e in epss:
        med = sy.Medium(base.n, base.h, base.lam0, base.mu0, base.rho0, base.dC * e, base.drho * e)
        F = op.FFTOperator(med, W10)
        x, *_ = solver.bicgstab(F.apply, u0, tol=1e-14, maxit=100)
        born = u0 + (u0 - F.apply(u0))
        errs.append(np.linalg.norm(x - born) / np.linalg.norm(u0))
    slope = np.log(errs[0] / errs[1]) / np.log(epss[0] / epss[1])
    assert 1.9 < slope < 2.1


def test_discrete_reciprocity():
    """With dC zero on boundary voxels the solution operator A^{-1} T is symmetric:
    the field at x_b (component j) from a unit force e_i at x_a equals the field at x_a
    (component i) from e_j at x_b."""
    med = sy.random_medium(6, seed=6, frac=0.15, zero_boundary=True)
    T = green.kernel_table(med.n, med.h, W10, med.lam0, med.mu0, med.rho0)
    F = op.FFTOperator(med, W10)
    xa, xb = (1, 2, 3), (4, 4, 2)
    for i, j in [(0, 1), (2, 2), (1, 0)]:
        ua, *_ = solver.bicgstab(F.apply, source.point_force_field(med.n, med.h, T, xa, i), tol=1e-14, maxit=200)
        ub, *_ = solver.bicgstab(F.apply, source.point_force_field(med.n, med.h, T, xb, j), tol=1e-14, maxit=200)
        l = ua[j, xb[2], xb[1], xb[0]]
        r = ub[i, xa[2], xa[1], xa[0]]
        assert abs(l - r) / abs(l) < 1e-10


def _navier_fd(u, C6, rho, h, w):
    """(c_ijkl u_k,l),j + rho w^2 u_i for constant c by 4th-order central differences (periodic roll)."""
    V = ((0, 5, 4), (5, 1, 3), (4, 3, 2))
    ax = lambda q: 2 - q  # noqa: E731

    def d1(f, a):
        return (-np.roll(f, -2, ax(a)) + 8 * np.roll(f, -1, ax(a)) - 8 * np.roll(f, 1, ax(a))
                + np.roll(f, 2, ax(a))) / (12 * h)

    def d2(f, a, b):
        if a == b:
            return (-np.roll(f, -2, ax(a)) + 16 * np.roll(f, -1, ax(a)) - 30 * f + 16 * np.roll(f, 1, ax(a))
                    - np.roll(f, 2, ax(a))) / (12 * h * h)
        return d1(d1(f, a), b)

    out = np.zeros_like(u)
    for i in range(3):
        acc = rho * w * w * u[i]
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    c = C6[V[i][j], V[k][l]]
                    if c != 0.0:
                        acc = acc + c * d2(u[k], j, l)
        out[i] = acc
    return out


@pytest.mark.slow
def test_solution_satisfies_wave_equation():
    """Eq. 1 pins the sign of every term: inside a uniform VTI + density contrast the LS solution
    satisfies the full medium's wave equation up to discretisation error, and does not satisfy the
    background's or the sign-flipped contrast's."""
    n, h = 24, 10.0
    lam, mu = sy.iso_lame(3000.0, 1730.0, 2300.0)
    C0 = sy.iso_voigt(lam, mu)
    dC6 = sy.thomsen_vti(3000.0, 1730.0, 2300.0, 0.1, 0.05, 0.08) - C0
    shape = (n, n, n)
    med = sy.Medium((n, n, n), h, lam, mu, 2300.0,
                    np.broadcast_to(sy.pack21(dC6)[:, None, None, None], (21,) + shape).copy(),
                    np.full(shape, 0.05 * 2300.0))
    w = 2 * np.pi * 8.0
    c = (n - 1) / 2
    u0, _ = source.background_field(med.n, h, sy.explosion(), np.array([c, c, c]) * h, w, lam, mu, 2300.0)
    x, it, rr, st, _ = solver.bicgstab(op.FFTOperator(med, w).apply, u0, tol=1e-10, maxit=200)
    assert st == 0
    b = 5
    sl = (slice(None),) + (slice(b, n - b),) * 3
    Z, Y, X = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    mask = (np.sqrt((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) > 6)[b:n - b, b:n - b, b:n - b]
    res = {}
    for name, C6, rho in [("true", C0 + dC6, 2300 * 1.05), ("flip", C0 - dC6, 2300 * 0.95), ("bg", C0, 2300.0)]:
        R = _navier_fd(x, C6, rho, h, w)[sl][:, mask]
        res[name] = np.linalg.norm(R) / np.linalg.norm(rho * w * w * np.abs(x[sl][:, mask]))
    assert res["true"] < 0.08
    assert res["true"] < 0.3 * res["bg"]
    assert res["true"] < 0.15 * res["flip"]


def test_apply_at_points_equals_fft_form():
    """The pointwise direct-sum evaluation used for full-size GPU checks agrees with the FFT form."""
    med = sy.random_medium((7, 6, 9), h=8.0, seed=13, frac=0.2)
    u = _field(med.shape, 14)
    full = op.FFTOperator(med, W10).apply(u)
    pts = [(0, 0, 0), (6, 5, 8), (3, 2, 4), (1, 5, 0)]
    got = op.apply_at_points(u, med, W10, pts)
    for (ix, iy, iz), g in zip(pts, got):
        assert np.abs(g - full[:, iz, iy, ix]).max() < 1e-13 * np.abs(full).max()


def test_taper_weight_properties():
    """Eq. 25's weight: zero on the outer node planes, 1 beyond the layer, symmetric, separable,
    increasing inward, and 1 - exp(-l^2 / (N h^2)) on a single-axis profile."""
    n, h, width = (20, 12, 16), 7.0, 5
    w = op.taper_weight(n, h, width)
    assert w.shape == (16, 12, 20)
    assert np.all(w[0] == 0) and np.all(w[:, :, -1] == 0) and np.all(w[:, 0, :] == 0)
    assert np.all(w[5:-5, 5:-5, 5:-5] == 1.0)
    assert np.allclose(w, w[::-1, ::-1, ::-1])
    prof = w[8, 6, :]
    assert np.all(np.diff(prof[:6]) > 0) and prof[5] == 1.0
    # Eq. 25 along x (N_x = 20 nodes, node k at distance l = k h from the outer plane): the weight
    # is 1 - exp(-k^2 / 20), worked out by hand from e^-0.05, e^-0.2, e^-0.45, e^-0.8
    hand = [0.0, 0.048770575499286, 0.181269246922018, 0.362371848378227, 0.550671035882778]
    assert np.allclose(prof[:5], hand, rtol=0, atol=1e-14)
    # separable: w = w_x w_y w_z
    assert np.allclose(w[2, 3, 4], w[2, 6, 10] * w[8, 3, 10] * w[8, 6, 4])
    assert np.array_equal(op.taper_weight(n, h, 0), np.ones((16, 12, 20)))


def test_taper_zeroes_boundary_contrast_sources():
    """With the taper a contrast that touches the boundary contributes nothing on the outer planes:
    the operator equals that of the medium whose boundary-node contrast is zero there."""
    med = sy.random_medium((8, 7, 9), h=10.0, seed=61, frac=0.2)
    t = op.tapered(med, 3)
    assert np.all(t.dC[:, 0] == 0) and np.all(t.drho[:, :, -1] == 0)
    assert np.allclose(t.dC[:, 4, 3, 4], med.dC[:, 4, 3, 4])
    u = _field(med.shape, 62)
    a = op.FFTOperator(t, W10).apply(u)
    b = (op.dense_matrix(t, W10) @ u.reshape(-1)).reshape(u.shape)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-13
