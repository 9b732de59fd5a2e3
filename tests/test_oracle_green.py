"""Pins of the oracle's Green's tensor, its derivative, the self-cell value and the kernel table.

Each check ties the oracle to something other than itself: Kelvin's static
solution, the PDE of Eq. 7 by finite differences, Richardson extrapolation,
a surface-integral quadrature, symmetry.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import green

LAM, MU, RHO = 2300.0 * (3000.0 ** 2 - 2 * 1730.0 ** 2), 2300.0 * 1730.0 ** 2, 2300.0
ALPHA, BETA = 3000.0, 1730.0


def _pts(k=7, scale=30.0, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((k, 3)) * scale


def _kelvin(x):
    """Kelvin's static point-force solution (textbook closed form)."""
    r = np.linalg.norm(x, axis=-1)
    g = x / r[:, None]
    gg = g[:, :, None] * g[:, None, :]
    return ((LAM + 3 * MU) * np.eye(3) + (LAM + MU) * gg) / (8 * np.pi * MU * (LAM + 2 * MU) * r[:, None, None])


def test_speeds():
    a, b = green.speeds(LAM, MU, RHO)
    assert a == pytest.approx(ALPHA, rel=1e-12)
    assert b == pytest.approx(BETA, rel=1e-12)


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_static_limit_is_kelvin(mode):
    x = _pts()
    K = _kelvin(x)
    G = green.green(x, 1e-2, LAM, MU, RHO, mode)
    # real part: Kelvin to O((w r / c)^2); the imaginary part is O(w) and isotropic-free of 1/r
    assert np.abs(G.real - K).max() / np.abs(K).max() < 1e-6


def test_exact_first_dynamic_term():
    """G_exact = Kelvin + i w (1/(3 a^3) + 2/(3 b^3)) I / (4 pi rho) + O(w^2 r)."""
    x = _pts(scale=20.0)
    K = _kelvin(x)
    c1 = (1 / (3 * ALPHA ** 3) + 2 / (3 * BETA ** 3)) / (4 * np.pi * RHO)
    rem = []
    for w in (1.0, 2.0):
        G = green.green(x, w, LAM, MU, RHO, "exact")
        rem.append(np.abs(G - K - 1j * w * c1 * np.eye(3)).max())
    # remainder is second order in w: doubling w multiplies it by ~4
    assert 3.5 < rem[1] / rem[0] < 4.5
    assert rem[0] / np.abs(K).max() < 1e-4


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_symmetry(mode):
    x = _pts()
    G = green.green(x, 2 * np.pi * 10, LAM, MU, RHO, mode)
    Gm = green.green(-x, 2 * np.pi * 10, LAM, MU, RHO, mode)
    assert np.allclose(G, np.swapaxes(G, -1, -2), rtol=0, atol=1e-14 * np.abs(G).max())
    assert np.allclose(G, Gm, rtol=0, atol=1e-14 * np.abs(G).max())


def _navier_residual(fn, x0, w, hstep):
    """Background Navier operator of Eq. 7 applied to column n of G by 4th-order finite differences."""
    lam, mu = LAM, MU

    def G(x):
        return fn(x[None, :])[0]

    def d2(a, b):
        e = np.eye(3)
        if a == b:
            s = [(-1, 2), (16, 1), (-30, 0), (16, -1), (-1, -2)]
            return sum(c * G(x0 + k * hstep * e[a]) for c, k in s) / (12 * hstep ** 2)

        def d1(y, ax):
            return (-G(y + 2 * hstep * e[ax]) + 8 * G(y + hstep * e[ax]) - 8 * G(y - hstep * e[ax])
                    + G(y - 2 * hstep * e[ax])) / (12 * hstep)
        cs = [(-1, 2), (8, 1), (-8, -1), (1, -2)]
        return sum(c * d1(x0 + k * hstep * e[a], b) for c, k in cs) / (12 * hstep)

    H = [[d2(a, b) for b in range(3)] for a in range(3)]   # H[a][b][i, n] = d_a d_b G_in
    lap = H[0][0] + H[1][1] + H[2][2]
    graddiv = np.array([[sum(H[i][k][k, n] for k in range(3)) for n in range(3)] for i in range(3)])
    L = (lam + mu) * graddiv + mu * lap + RHO * w * w * G(x0)
    scale = np.abs(RHO * w * w * G(x0)).max() + np.abs(mu * lap).max()
    return np.abs(L).max() / scale


def test_exact_solves_navier():
    """Away from r = 0 the exact tensor satisfies (c0 G_kn,l),j + rho0 w^2 G_in = 0 (Eq. 7)."""
    w = 2 * np.pi * 15
    x0 = np.array([40.0, -25.0, 30.0])
    fn = lambda x: green.green(x, w, LAM, MU, RHO, "exact")  # noqa: E731
    e1 = _navier_residual(fn, x0, w, 1.0)
    e2 = _navier_residual(fn, x0, w, 0.5)
    assert e1 < 1e-6
    assert e2 < e1 / 8  # 4th order convergence
    # the paper's NF+FF form is not an exact solution: its residual does not vanish
    fp = lambda x: green.green(x, w, LAM, MU, RHO, "paper")  # noqa: E731
    assert _navier_residual(fp, x0, w, 0.5) > 1e-3


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_derivative_richardson(mode):
    x = _pts(scale=25.0, seed=3)
    w = 2 * np.pi * 12
    dG = green.dgreen(x, w, LAM, MU, RHO, mode)
    for k in range(3):
        def fd(s):
            e = np.zeros(3)
            e[k] = s
            return (green.green(x + e, w, LAM, MU, RHO, mode) - green.green(x - e, w, LAM, MU, RHO, mode)) / (2 * s)
        rich = (4 * fd(5e-3) - fd(1e-2)) / 3
        assert np.abs(rich - dG[..., k]).max() / np.abs(dG).max() < 1e-9


def test_paper_minus_exact_far_field():
    """Far from the source the exact tensor is the Eq. A.5 far field plus O(1/(k r^2)) terms.

    The paper's G keeps the static near-field term of Eq. A.4 (which decays
    like 1/r, as fast as the far field) at every distance, so
    G_paper - G_exact -> G^NF, with a remainder O(1/(k r)) relative.
    """
    w = 2 * np.pi * 40
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    for r in (200.0, 2000.0, 20000.0):
        x = (d * r)[None, :]
        Ge = green.green(x, w, LAM, MU, RHO, "exact")
        Gp = green.green(x, w, LAM, MU, RHO, "paper")
        g = d[:, None] * d[None, :]
        g_nf = -(1 - BETA ** 2 / ALPHA ** 2) / (8 * np.pi * RHO * r * BETA ** 2) * (np.eye(3) - 3 * g)
        err = np.abs(Gp - Ge - g_nf).max() / np.abs(Ge).max()
        # |3 g g - I| <= 2 bounds the intermediate term by 2 (1 + beta/alpha) / (k_beta r)
        assert err < 2 * (1 + BETA / ALPHA) / (w / BETA * r)
        # while the static term itself stays a fixed fraction of the far field
        assert np.abs(g_nf).max() / np.abs(Ge).max() > 0.2


def test_self_cell_constant_quadrature():
    """C = int over the unit cube of 1/|x| dV, by the divergence theorem as a smooth surface integral.

    div(x/|x|) = 2/|x|, so C = 1/2 * (surface integral of x.n/|x|) = 3 * int_{[-1/2,1/2]^2} (1/2)/sqrt(1/4+y^2+z^2).
    """
    val, _ = integrate.dblquad(lambda z, y: 0.5 / np.sqrt(0.25 + y * y + z * z), -0.5, 0.5, -0.5, 0.5,
                               epsabs=1e-14, epsrel=1e-14)
    assert 3.0 * val == pytest.approx(green.SELF_CELL_C, rel=1e-12)


def _cube_average(fn, h, order=24):
    """int over [-h/2, h/2]^3 of fn(x) dV, split into 6 face pyramids (integrand regular there)."""
    t, wt = np.polynomial.legendre.leggauss(order)
    tt = 0.5 * (t + 1.0)
    wt_t = 0.5 * wt
    T, S1, S2 = np.meshgrid(tt, t, t, indexing="ij")
    W = wt_t[:, None, None] * wt[None, :, None] * wt[None, None, :]
    total = 0.0
    for ax in range(3):
        for sgn in (1.0, -1.0):
            pts = np.zeros(T.shape + (3,))
            others = [a for a in range(3) if a != ax]
            pts[..., ax] = sgn * T * h / 2
            pts[..., others[0]] = S1 * T * h / 2
            pts[..., others[1]] = S2 * T * h / 2
            jac = (h / 2) ** 3 * T ** 2
            vals = fn(pts.reshape(-1, 3)).reshape(T.shape + (3, 3))
            total = total + np.sum((W * jac)[..., None, None] * vals, axis=(0, 1, 2))
    return total


def test_self_cell_is_cell_average():
    h = 10.0
    for f in (2.0, 5.0):
        w = 2 * np.pi * f
        num = _cube_average(lambda x: green.green(x, w, LAM, MU, RHO, "exact"), h)
        ref = green.self_cell(h, w, LAM, MU, RHO)
        kh = w * h / BETA
        # formula keeps terms to O(w h); the remainder is O((w h / beta)^2) relative
        assert np.abs(num - ref).max() / np.abs(ref).max() < 0.5 * kh ** 2
        # the off-diagonal average vanishes by symmetry
        assert np.abs(num - np.diag(np.diag(num))).max() < 1e-12 * np.abs(num).max()


def test_kernel_table_layout():
    n = (4, 3, 5)
    h = 7.0
    w = 2 * np.pi * 9
    T = green.kernel_table(n, h, w, LAM, MU, RHO)
    assert T.shape == (3, 3, 10, 6, 8)
    # Nyquist planes m_a = n_a are zero
    assert np.all(T[:, :, :, :, 4] == 0) and np.all(T[:, :, :, 3, :] == 0) and np.all(T[:, :, 5] == 0)
    # an offset (mx, my, mz) = (-3, 2, 1) sits at index (mz, my, mx mod 8) and equals h^3 G(m h)
    G = green.green(np.array([[-3 * h, 2 * h, 1 * h]]), w, LAM, MU, RHO)[0] * h ** 3
    assert np.allclose(T[:, :, 1, 2, 5], G, rtol=1e-14, atol=0)
    assert np.allclose(T[:, :, 0, 0, 0], green.self_cell(h, w, LAM, MU, RHO))
    # kernel is even: T(m) = T(-m)
    Tm = T[:, :, (-np.arange(10)) % 10][:, :, :, (-np.arange(6)) % 6][:, :, :, :, (-np.arange(8)) % 8]
    assert np.allclose(T, Tm, rtol=1e-14, atol=1e-30)
