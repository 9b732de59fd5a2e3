"""Moment-tensor sources in Voigt order (M11, M22, M33, M23, M13, M12) (Sec. 2.1)."""
from __future__ import annotations

import numpy as np


def voigt_moment(M3):
    """3x3 symmetric moment tensor -> Voigt 6-vector (11, 22, 33, 23, 13, 12)."""
    M3 = np.asarray(M3, dtype=float)
    return np.array([M3[0, 0], M3[1, 1], M3[2, 2], M3[1, 2], M3[0, 2], M3[0, 1]])


def explosion(scale=1.0):
    return voigt_moment(np.eye(3) * scale)


def clvd():
    return voigt_moment(np.diag([-1.0, -1.0, 2.0]) / np.sqrt(6.0))


def double_couple_12():
    """Strike-slip double couple, M12 = M21 = 1/sqrt(2) (Table 1)."""
    M = np.zeros((3, 3))
    M[0, 1] = M[1, 0] = 1.0 / np.sqrt(2.0)
    return voigt_moment(M)


def double_couple_13():
    """Dip-slip double couple, M13 = M31 = 1/sqrt(2) (Table 3)."""
    M = np.zeros((3, 3))
    M[0, 2] = M[2, 0] = 1.0 / np.sqrt(2.0)
    return voigt_moment(M)


def random_moment_tensors(k, rng):
    """k random symmetric moment tensors, 6 iid N(0,1) entries, unit Frobenius norm."""
    out = []
    for _ in range(k):
        a = rng.standard_normal(6)
        M = np.array([[a[0], a[5], a[4]], [a[5], a[1], a[3]], [a[4], a[3], a[2]]])
        M /= np.linalg.norm(M)
        out.append(voigt_moment(M))
    return np.array(out)
