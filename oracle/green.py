"""Background elastodynamic Green's tensor (Eq. 7, Appendix A).  FP64, NumPy.

Test infrastructure: part of the CPU oracle (see ``oracle/__init__.py``).

Conventions (readings of the paper):

* time dependence exp(-i w t), so outgoing waves are exp(+i w r / c)
  (the far-field terms of Eq. A.5);
* G_ij(x) is the i-displacement at offset x = receiver - source from a unit
  force along j; it solves Eq. 7 with the background density rho0;
* two closed forms are provided:
  - ``mode="exact"``: the full isotropic solution of Eq. 7 (near, intermediate
    and far field), whose static limit is Kelvin's solution;
  - ``mode="paper"``: the paper's G = G^NF (Eq. A.4) + G^FF (Eq. A.5), with
    its derivatives from Eqs. A.6-A.11.
"""
from __future__ import annotations

import numpy as np

EYE = np.eye(3)


def speeds(lam, mu, rho):
    """P and S velocities (alpha, beta) of the isotropic background."""
    return np.sqrt((lam + 2.0 * mu) / rho), np.sqrt(mu / rho)


def _geometry(x):
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(np.sum(x * x, axis=-1))
    xx = x[..., :, None] * x[..., None, :]                       # x_i x_j
    # T1[i,j,k] = d_ik x_j + d_jk x_i ; T3[i,j,k] = x_i x_j x_k
    T1 = EYE[:, None, :] * x[..., None, :, None] + EYE[None, :, :] * x[..., :, None, None]
    T3 = xx[..., :, :, None] * x[..., None, None, :]
    return x, r, xx, T1, T3


def green(x, omega, lam, mu, rho, mode="exact"):
    """G_ij(x) for offsets x of shape (..., 3), |x| > 0.  Returns (..., 3, 3) complex."""
    alpha, beta = speeds(lam, mu, rho)
    x, r, xx, _, _ = _geometry(x)
    R = r[..., None, None]
    Y = xx / R ** 2                                               # x_i x_j / r^2
    ka, kb = omega / alpha, omega / beta
    ea = np.exp(1j * ka * r)[..., None, None]
    eb = np.exp(1j * kb * r)[..., None, None]
    g_p = ea * Y / (4.0 * np.pi * rho * alpha ** 2 * R)           # Eq. A.5, P term
    g_s = eb * (EYE - Y) / (4.0 * np.pi * rho * beta ** 2 * R)    # Eq. A.5, S term
    if mode == "paper":
        c_nf = (1.0 - beta ** 2 / alpha ** 2) / (8.0 * np.pi * rho * beta ** 2)
        g_n = -c_nf * (EYE - 3.0 * Y) / R                         # Eq. A.4
    elif mode == "exact":
        rr = r[..., None, None]
        phi = ((1.0 - 1j * kb * rr) * eb - (1.0 - 1j * ka * rr) * ea)
        g_n = (3.0 * Y - EYE) * phi / (4.0 * np.pi * rho * omega ** 2 * rr ** 3)
    else:
        raise ValueError(mode)
    return g_p + g_s + g_n


def dgreen(x, omega, lam, mu, rho, mode="exact"):
    """dG_ij/dx_k at offsets x (..., 3).  Returns (..., 3, 3, 3) complex, index [i, j, k].

    Product-rule form of Appendix A: each term is written as a radial factor
    times a direction tensor, as in Eqs. A.6-A.11.
    """
    alpha, beta = speeds(lam, mu, rho)
    x, r, xx, T1, T3 = _geometry(x)
    U = r[..., None, None, None]                                  # U = r
    Uk = (x / r[..., None])[..., None, None, :]                   # U_,k = x_k / r
    Y = (xx / (r ** 2)[..., None, None])[..., None]               # Y_ij (broadcast over k)
    Yk = (U ** 2 * T1 - 2.0 * T3) / U ** 4                        # Y_ij,k
    ka, kb = omega / alpha, omega / beta
    rr = r[..., None, None, None]
    xk = x[..., None, None, :]

    # P term (Eqs. A.8-A.9): X(r) Y_ij / U
    X = np.exp(1j * ka * rr) / (4.0 * np.pi * rho * alpha ** 2)
    Xk = 1j * omega * X * xk / (alpha * rr)
    d_p = ((Xk * Y + X * Yk) * U - X * Y * Uk) / U ** 2
    # S term (Eqs. A.10-A.11): V(r) W_ij / U, W = I - Y
    V = np.exp(1j * kb * rr) / (4.0 * np.pi * rho * beta ** 2)
    Vk = 1j * omega * V * xk / (beta * rr)
    W = EYE[..., None] - Y
    Wk = -Yk
    d_s = ((Vk * W + V * Wk) * U - V * W * Uk) / U ** 2

    if mode == "paper":
        # Eqs. A.6-A.7: G^NF = -C E / U, E = I - 3 x x^T / r^2
        C = (1.0 - beta ** 2 / alpha ** 2) / (8.0 * np.pi * rho * beta ** 2)
        E = EYE[..., None] - 3.0 * Y
        D = xk
        F = xx[..., None]
        d_n = C / U ** 3 * (D * E - 3.0 / U ** 2 * (2.0 * F * D - T1 * U ** 2))
    elif mode == "exact":
        # near/intermediate term Z(r) (3 Y_ij - d_ij), Z = Phi(r) / (4 pi rho w^2 r^3),
        # Phi = (1 - i kb r) e^{i kb r} - (1 - i ka r) e^{i ka r}
        ea = np.exp(1j * ka * rr)
        eb = np.exp(1j * kb * rr)
        phi = (1.0 - 1j * kb * rr) * eb - (1.0 - 1j * ka * rr) * ea
        dphi = rr * (kb ** 2 * eb - ka ** 2 * ea)
        c = 1.0 / (4.0 * np.pi * rho * omega ** 2)
        Z = c * phi / rr ** 3
        Zr = c * (dphi / rr ** 3 - 3.0 * phi / rr ** 4)
        d_n = Zr * Uk * (3.0 * Y - EYE[..., None]) + Z * 3.0 * Yk
    else:
        raise ValueError(mode)
    return d_p + d_s + d_n


SELF_CELL_C = 3.0 * np.log(2.0 + np.sqrt(3.0)) - np.pi / 2.0   # int_{[-1/2,1/2]^3} dV/|x|


def self_cell(h, omega, lam, mu, rho):
    """Cube average of G over the cell [-h/2, h/2]^3 times h^3, to O(w h).

    Expanding G for small r: the static Kelvin part averages to
    (1/(3 alpha^2) + 2/(3 beta^2)) / (4 pi rho) * delta_ij * int dV / r, the
    near-field (3 g g - I) part averages to zero over a cube, and the O(r^0)
    term of exp(i k r)/r leaves i w (1/(3 alpha^3) + 2/(3 beta^3)) delta_ij /
    (4 pi rho).  The same two numbers come out of Eq. A.4 + A.5, so both
    modes share this value.
    """
    alpha, beta = speeds(lam, mu, rho)
    static = (1.0 / (3.0 * alpha ** 2) + 2.0 / (3.0 * beta ** 2)) * SELF_CELL_C * h * h
    dyn = 1j * omega * (1.0 / (3.0 * alpha ** 3) + 2.0 / (3.0 * beta ** 3)) * h ** 3
    return (static + dyn) / (4.0 * np.pi * rho) * EYE


def kernel_table(n, h, omega, lam, mu, rho, mode="exact"):
    """Sampled kernel on the 2n-periodic grid, shape (3, 3, 2nz, 2ny, 2nx) complex.

    Entry [i, j, mz, my, mx] holds h^3 G_ij(m h) for the signed offset m whose
    components satisfy |m_a| <= n_a - 1 (m != 0), the self-cell value at m = 0,
    and zero on the planes m_a = n_a (the offset that a 2n-periodic grid
    cannot tell apart from -n_a).  Index m_a maps to m_a mod 2 n_a.
    """
    nx, ny, nz = n
    T = np.zeros((3, 3, 2 * nz, 2 * ny, 2 * nx), dtype=np.complex128)
    mx = np.arange(-(nx - 1), nx)
    my = np.arange(-(ny - 1), ny)
    mz = np.arange(-(nz - 1), nz)
    MZ, MY, MX = np.meshgrid(mz, my, mx, indexing="ij")
    off = np.stack([MX, MY, MZ], axis=-1).astype(np.float64) * h
    zero = (MX == 0) & (MY == 0) & (MZ == 0)
    off[zero] = 1.0  # placeholder, overwritten below
    G = green(off, omega, lam, mu, rho, mode) * h ** 3
    G[zero] = self_cell(h, omega, lam, mu, rho)
    G = np.moveaxis(G, (-2, -1), (0, 1))              # (3, 3, z, y, x)
    T[:, :, MZ % (2 * nz), MY % (2 * ny), MX % (2 * nx)] = G
    return T


def h_table(n, h, omega, lam, mu, rho, mode="exact"):
    """Sampled derivative kernel of Eqs. 9-10 on the 2n-periodic grid, shape (3, 6, 2nz, 2ny, 2nx).

    Entry [i, J, m] is the weight of the Voigt stress sigma_J in u_s,i = sum_jk (dG_ij/dx_k) * sigma_jk
    (Eq. 8 after partial integration): h^3 dG_ij/dx_k (m h) for J = (j, j), and
    h^3 (dG_ij/dx_k + dG_ik/dx_j)(m h) for J = (j, k), j != k (both orderings of the symmetric
    stress).  Zero at m = 0 (the cell average of an odd function) and on the planes m_a = n_a;
    index layout as in ``kernel_table``.
    """
    nx, ny, nz = n
    T = np.zeros((3, 6, 2 * nz, 2 * ny, 2 * nx), dtype=np.complex128)
    mx = np.arange(-(nx - 1), nx)
    my = np.arange(-(ny - 1), ny)
    mz = np.arange(-(nz - 1), nz)
    MZ, MY, MX = np.meshgrid(mz, my, mx, indexing="ij")
    off = np.stack([MX, MY, MZ], axis=-1).astype(np.float64) * h
    zero = (MX == 0) & (MY == 0) & (MZ == 0)
    off[zero] = 1.0  # placeholder, zeroed below
    dG = dgreen(off, omega, lam, mu, rho, mode) * h ** 3            # (z, y, x, i, j, k)
    dG[zero] = 0.0
    voigt = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    for J, (j, k) in enumerate(voigt):
        w = dG[..., :, j, k] if j == k else dG[..., :, j, k] + dG[..., :, k, j]
        T[:, J][:, MZ % (2 * nz), MY % (2 * ny), MX % (2 * nx)] = np.moveaxis(w, -1, 0)
    return T
