"""Background field of a moment-tensor point source (Eqs. 13-16).  FP64, NumPy.

Test infrastructure: part of the CPU oracle (see ``oracle/__init__.py``).

With the body force f_i = -M_ij d/dx_j delta(x - s) (Eq. 13, rupture time
t0 = 0) in the convolution of Eq. 6, moving the derivative off the delta
gives u0_i(x) = M_jk dG_ij(x, xi)/d xi_k at xi = s, and because G depends on
x - xi only, u0_i(x) = -M_jk (dG_ij/dx_k)(x - s).  Eq. 15 writes this with
H; we read its H as the derivative with respect to the source coordinate.

A node that coincides with the source gets u0 = 0 there (the cell average of
an odd function of x - s) and the call reports it.
"""
from __future__ import annotations

import numpy as np

from . import green as _green


def moment_3x3(M6):
    """Voigt (11, 22, 33, 23, 13, 12) -> symmetric 3x3."""
    m = np.asarray(M6, dtype=np.float64)
    return np.array([[m[0], m[5], m[4]], [m[5], m[1], m[3]], [m[4], m[3], m[2]]])


def background_field(n, h, M6, xs, omega, lam, mu, rho, mode="exact"):
    """u0 (3, nz, ny, nx) complex on the model's nodes, and whether a node hit the source."""
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz) * h, np.arange(ny) * h, np.arange(nx) * h, indexing="ij")
    off = np.stack([X - xs[0], Y - xs[1], Z - xs[2]], axis=-1)
    r = np.sqrt(np.sum(off * off, axis=-1))
    on_node = r == 0.0
    off[on_node] = 1.0
    dG = _green.dgreen(off, omega, lam, mu, rho, mode)          # [..., i, j, k]
    M = moment_3x3(M6)
    u0 = -np.einsum("...ijk,jk->i...", dG, M)
    u0[:, on_node] = 0.0
    return u0, bool(on_node.any())


def point_force_field(n, h, table, node, comp):
    """Oracle-only helper: u0 = T(x - x_node) e_comp, the table column of a unit force on a node."""
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mz = (Z - node[2]) % (2 * nz)
    my = (Y - node[1]) % (2 * ny)
    mx = (X - node[0]) % (2 * nx)
    return np.stack([table[i, comp][mz, my, mx] for i in range(3)])


def moment_gradient(lam, n, h, xs, omega, lam0, mu0, rho0, mode="exact"):
    """Re<lam, d u0 / d M_J> for the six Voigt components (u0 is linear in M, Eqs. 13-16)."""
    out = np.zeros(6)
    for J in range(6):
        e = np.zeros(6)
        e[J] = 1.0
        u0, _ = background_field(n, h, e, xs, omega, lam0, mu0, rho0, mode)
        out[J] = np.real(np.vdot(lam, u0))
    return out
