"""Synthetic media: isotropic background + Voigt stiffness contrast + density contrast.

Layout conventions (shared by every consumer of these arrays):

* grid node (ix, iy, iz) sits at (ix*h, iy*h, iz*h) metres;
* scalar fields are float64 arrays of shape (nz, ny, nx), x fastest;
* the stiffness contrast is 21 planes, shape (21, nz, ny, nx): the upper
  triangle of the symmetric 6x6 Voigt matrix, row-major
  (1,1),(1,2),...,(1,6),(2,2),...,(2,6),...,(6,6), Voigt order
  11, 22, 33, 23, 13, 12 (Sec. 3.1);
* stiffnesses in Pa, densities in kg/m^3.

Everything here is input construction only (Thomsen's VTI parameters, Bond
rotation, Gaussian random fields).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2301_12836

GPA = 1.0e9


@dataclass
class Medium:
    """A homogeneous isotropic background (lam0, mu0, rho0) plus contrasts."""

    n: tuple            # (nx, ny, nz)
    h: float            # grid spacing [m]
    lam0: float         # background Lame lambda [Pa]
    mu0: float          # background shear modulus [Pa]
    rho0: float         # background density [kg/m^3]
    dC: np.ndarray      # (21, nz, ny, nx) float64, stiffness contrast [Pa]
    drho: np.ndarray    # (nz, ny, nx) float64, density contrast [kg/m^3]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    @property
    def vp0(self):
        return float(np.sqrt((self.lam0 + 2.0 * self.mu0) / self.rho0))

    @property
    def vs0(self):
        return float(np.sqrt(self.mu0 / self.rho0))


def iso_lame(vp, vs, rho):
    """Lame parameters of an isotropic medium from its velocities and density."""
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def iso_voigt(lam, mu):
    """6x6 Voigt stiffness of an isotropic medium."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    for i in range(3):
        C[i, i] = lam + 2.0 * mu
        C[3 + i, 3 + i] = mu
    return C


def thomsen_vti(vp0, vs0, rho, eps, delta, gamma):
    """VTI stiffness from vertical velocities and Thomsen's (1986) parameters."""
    c33 = rho * vp0 * vp0
    c44 = rho * vs0 * vs0
    c11 = c33 * (1.0 + 2.0 * eps)
    c66 = c44 * (1.0 + 2.0 * gamma)
    c13 = np.sqrt(2.0 * delta * c33 * (c33 - c44) + (c33 - c44) ** 2) - c44
    c12 = c11 - 2.0 * c66
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = c11
    C[2, 2] = c33
    C[0, 1] = C[1, 0] = c12
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = c13
    C[3, 3] = C[4, 4] = c44
    C[5, 5] = c66
    return C


def _bond_matrix(R):
    """6x6 Bond stress-transformation matrix for a 3x3 rotation R (Voigt 11,22,33,23,13,12)."""
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    M = np.zeros((6, 6))
    for I, (i, j) in enumerate(pairs):
        for J, (k, l) in enumerate(pairs):
            if J < 3:
                M[I, J] = R[i, k] * R[j, l]
            else:
                M[I, J] = R[i, k] * R[j, l] + R[i, l] * R[j, k]
    return M


def bond_rotate_y(C, tilt_rad):
    """Rotate a Voigt stiffness about the y axis by tilt_rad (tilted TI media)."""
    c, s = np.cos(tilt_rad), np.sin(tilt_rad)
    R = np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])
    M = _bond_matrix(R)
    return M @ C @ M.T


_TRIU = [(I, J) for I in range(6) for J in range(I, 6)]


def pack21(C):
    """Upper triangle of a symmetric 6x6 (or 6x6xgrid) Voigt array, row-major."""
    return np.stack([C[I, J] for I, J in _TRIU])


def unpack21(c21):
    """Inverse of pack21 (symmetric 6x6 from 21 planes)."""
    c21 = np.asarray(c21)
    C = np.zeros((6, 6) + c21.shape[1:], dtype=c21.dtype)
    for k, (I, J) in enumerate(_TRIU):
        C[I, J] = c21[k]
        C[J, I] = c21[k]
    return C


def gaussian_random_field(shape, h, corr_len, rng):
    """Zero-mean unit-std field with Gaussian covariance exp(-r^2/L^2).

    White N(0,1) noise filtered in k-space by the square root of the
    covariance's spectrum, then renormalised to unit standard deviation.
    """
    white = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(s, d=h) * 2.0 * np.pi for s in shape]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    # spectrum of exp(-r^2/L^2) is proportional to exp(-k^2 L^2 / 4)
    filt = np.exp(-k2 * corr_len * corr_len / 8.0)
    f = np.fft.ifftn(np.fft.fftn(white) * filt).real
    f -= f.mean()
    f /= f.std()
    return f


def _grid_of(C6, shape):
    return np.broadcast_to(pack21(C6)[:, None, None, None], (21,) + tuple(shape)).copy()


def inclusion_medium(n=16, h=10.0, vp=3000.0, vs=1730.0, rho=2300.0,
                     eps=0.1, delta=0.05, gamma=0.08, drho_frac=0.05, lo=None, hi=None):
    """Isotropic background with a centred cube of VTI material (Thomsen) and +5% density.

    Default: 16^3 nodes, 10 m spacing, inclusion on nodes 5..10 of every axis
    (a 6^3 cube), so the contrast vanishes on the boundary planes.
    """
    lam, mu = iso_lame(vp, vs, rho)
    lo = (n - 6) // 2 if lo is None else lo
    hi = lo + 6 if hi is None else hi
    dC6 = thomsen_vti(vp, vs, rho, eps, delta, gamma) - iso_voigt(lam, mu)
    shape = (n, n, n)
    dC = np.zeros((21,) + shape)
    drho = np.zeros(shape)
    sl = (slice(lo, hi),) * 3
    d21 = pack21(dC6)
    for k in range(21):
        dC[k][sl] = d21[k]
    drho[sl] = drho_frac * rho
    return Medium((n, n, n), h, lam, mu, rho, dC, drho, name=f"vti_inclusion_{n}",
                  meta=dict(vp=vp, vs=vs, inclusion=(lo, hi), eps=eps, delta=delta, gamma=gamma))


def layered_vti_medium(n=64, h=10.0, rho=2300.0, seed_offset=2):
    """Three horizontal VTI layers (vp 2500/3000/3500, vs = vp/sqrt(3)) over a 3000 m/s background.

    Thomsen (eps, delta, gamma) per layer drawn from U[0, 0.2], seeded.
    """
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    vp0, vs0 = 3000.0, 3000.0 / np.sqrt(3.0)
    lam, mu = iso_lame(vp0, vs0, rho)
    C0 = iso_voigt(lam, mu)
    bounds = [0, round(n / 3), round(2 * n / 3), n]
    vps = [2500.0, 3000.0, 3500.0]
    shape = (n, n, n)
    dC = np.zeros((21,) + shape)
    params = []
    for L in range(3):
        e, d, g = rng.uniform(0.0, 0.2, size=3)
        C = thomsen_vti(vps[L], vps[L] / np.sqrt(3.0), rho, e, d, g)
        params.append((vps[L], e, d, g))
        d21 = pack21(C - C0)
        for k in range(21):
            dC[k, bounds[L]:bounds[L + 1]] = d21[k]
    drho = np.zeros(shape)
    return Medium((n, n, n), h, lam, mu, rho, dC, drho, name=f"vti_layers_{n}",
                  meta=dict(layers=params, bounds=bounds))


def grf_orthorhombic_medium(n=128, h=8.0, vp=3000.0, vs=1730.0, rho=2300.0,
                            std=0.05, corr_len=40.0, seed_offset=3):
    """Isotropic background + Gaussian-random-field orthorhombic contrast.

    Each of the 9 orthorhombic entries is perturbed by std * C0_IJ * g_IJ(x)
    with independent unit-std GRFs (correlation length corr_len); the other
    12 entries are stored as zeros.  Density: std * rho0 * g_rho(x).
    """
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    lam, mu = iso_lame(vp, vs, rho)
    C0 = iso_voigt(lam, mu)
    shape = (n, n, n)
    dC6 = np.zeros((6, 6) + shape)
    for I, J in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2), (3, 3), (4, 4), (5, 5)]:
        g = gaussian_random_field(shape, h, corr_len, rng)
        dC6[I, J] = std * C0[I, J] * g
        dC6[J, I] = dC6[I, J]
    drho = std * rho * gaussian_random_field(shape, h, corr_len, rng)
    return Medium((n, n, n), h, lam, mu, rho, pack21(dC6), drho, name=f"grf_ortho_{n}",
                  meta=dict(std=std, corr_len=corr_len))


# Table 2 of the paper (GPa): top VTI, isotropic, bottom VTI layers.
TABLE2 = {
    "top": dict(c11=34.0, c33=26.5, c55=10.4, c66=11.7, c13=6.9),
    "iso": dict(c11=29.05, c33=29.05, c55=10.0, c66=10.0, c13=9.05),
    "bottom": dict(c11=33.8, c33=21.9, c55=6.0, c66=12.0, c13=8.0),
}


def vti_from_table(c11, c33, c55, c66, c13):
    """6x6 VTI Voigt stiffness [Pa] from five coefficients [GPa], c12 = c11 - 2 c66."""
    C = np.zeros((6, 6))
    C[0, 0] = C[1, 1] = c11
    C[2, 2] = c33
    C[0, 1] = C[1, 0] = c11 - 2.0 * c66
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = c13
    C[3, 3] = C[4, 4] = c55
    C[5, 5] = c66
    return C * GPA


def table2_layers_medium(n=96, h=10.0, rho=2500.0, perturb=0.03, seed_offset=4, corr_len=40.0):
    """Three layers of Table 2 (VTI / isotropic / VTI) with a 3% GRF perturbation.

    The background is the isotropic layer (c11 = 29.05, c44 = 10.0 GPa).
    """
    rng = np.random.default_rng(BASE_SEED + seed_offset)
    iso = TABLE2["iso"]
    mu = iso["c55"] * GPA
    lam = iso["c11"] * GPA - 2.0 * mu
    C0 = iso_voigt(lam, mu)
    shape = (n, n, n)
    b = [0, n // 3, 2 * n // 3, n]
    dC6 = np.zeros((6, 6) + shape)
    for L, key in enumerate(["top", "iso", "bottom"]):
        C = vti_from_table(**TABLE2[key])
        dC6[:, :, b[L]:b[L + 1]] = C[:, :, None, None, None]
    if perturb:
        for I in range(6):
            for J in range(I, 6):
                if np.any(dC6[I, J] != 0.0):
                    g = gaussian_random_field(shape, h, corr_len, rng)
                    dC6[I, J] = dC6[I, J] * (1.0 + perturb * g)
                    dC6[J, I] = dC6[I, J]
    dC6 = dC6 - C0[:, :, None, None, None]
    drho = np.zeros(shape)
    return Medium((n, n, n), h, lam, mu, rho, pack21(dC6), drho, name=f"table2_layers_{n}",
                  meta=dict(bounds=b, perturb=perturb))


def tti_layer_medium(n=256, h=5.0, vp=3000.0, vs=1730.0, rho=2300.0,
                     eps=0.15, delta=0.1, gamma=0.12, tilt_deg=30.0, z0=None, z1=None):
    """Isotropic background with one tilted-TI (fractured) layer between isotropic layers."""
    lam, mu = iso_lame(vp, vs, rho)
    z0 = (3 * n) // 8 if z0 is None else z0
    z1 = (5 * n) // 8 if z1 is None else z1
    C = bond_rotate_y(thomsen_vti(vp, vs, rho, eps, delta, gamma), np.deg2rad(tilt_deg))
    d21 = pack21(C - iso_voigt(lam, mu))
    shape = (n, n, n)
    dC = np.zeros((21,) + shape)
    for k in range(21):
        dC[k, z0:z1] = d21[k]
    drho = np.zeros(shape)
    return Medium((n, n, n), h, lam, mu, rho, dC, drho, name=f"tti_layer_{n}",
                  meta=dict(z=(z0, z1), tilt_deg=tilt_deg))


def random_medium(n, h=10.0, vp=3000.0, vs=1730.0, rho=2300.0, frac=0.1, seed=0,
                  zero_boundary=False):
    """Small random full-anisotropy contrast (all 21 entries) for parity tests.

    n may be an int or an (nx, ny, nz) tuple.  Entries are uniform in
    [-frac, frac] times the background c11 (the 6x6 kept symmetric), density
    uniform in [-frac, frac] * rho.
    """
    rng = np.random.default_rng(BASE_SEED + 1000 + seed)
    nx, ny, nz = (n, n, n) if np.isscalar(n) else tuple(n)
    lam, mu = iso_lame(vp, vs, rho)
    shape = (nz, ny, nx)
    scale = lam + 2.0 * mu
    dC = rng.uniform(-frac, frac, size=(21,) + shape) * scale * 0.5
    drho = rng.uniform(-frac, frac, size=shape) * rho
    if zero_boundary:
        dC[:, [0, -1], :, :] = 0.0
        dC[:, :, [0, -1], :] = 0.0
        dC[:, :, :, [0, -1]] = 0.0
        drho[[0, -1], :, :] = 0.0
        drho[:, [0, -1], :] = 0.0
        drho[:, :, [0, -1]] = 0.0
    return Medium((nx, ny, nz), h, lam, mu, rho, dC, drho, name=f"random_{nx}x{ny}x{nz}")
