"""Pins of the oracle's sampled-H form of the operator (Eq. 21 with H of Eq. 9 sampled from the
analytic derivative of Appendix A) against things other than itself:

* the sampled table against central differences of the Green's tensor itself (not of dgreen),
  with the Voigt weights of Eq. 10 (both orderings of an off-diagonal stress);
* the parity of each entry under a mirrored axis (what an octant-folded spectrum relies on);
* the FFT evaluation against the brute-force direct sum on tiny grids;
* second-order agreement with the difference form (the default operator) on a smooth contrast:
  both discretise the same integral of Eq. 8, so their difference must fall like h^2.
"""
import numpy as np
import pytest

import synthetic as sy
from oracle import green as og, operator as op

RHO = 2300.0
LAM, MU = sy.iso_lame(3000.0, 1730.0, RHO)
W = 2 * np.pi * 9.0
VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_h_table_is_the_voigt_weighted_derivative_of_green(mode):
    n, h = (5, 4, 6), 7.0
    H = og.h_table(n, h, W, LAM, MU, RHO, mode)
    d = 1e-4 * h
    for m in [(1, 0, 0), (2, -1, 3), (-4, 3, -5), (0, -2, 1)]:
        x = np.array(m, dtype=np.float64) * h
        dG = np.zeros((3, 3, 3), dtype=np.complex128)   # [i, j, k] = dG_ij / dx_k by central differences
        for k in range(3):
            e = np.zeros(3)
            e[k] = d
            dG[:, :, k] = (og.green(x + e, W, LAM, MU, RHO, mode) - og.green(x - e, W, LAM, MU, RHO, mode)) / (2 * d)
        idx = (m[2] % (2 * n[2]), m[1] % (2 * n[1]), m[0] % (2 * n[0]))
        for J, (j, k) in enumerate(VOIGT):
            want = dG[:, j, k] if j == k else dG[:, j, k] + dG[:, k, j]
            got = H[(slice(None), J) + idx] / h ** 3
            assert np.abs(got - want).max() <= 1e-6 * np.abs(dG).max()
    assert np.all(H[:, :, 0, 0, 0] == 0)                       # odd kernel: zero cell average
    assert np.all(H[:, :, n[2]] == 0) and np.all(H[:, :, :, n[1]] == 0) and np.all(H[:, :, :, :, n[0]] == 0)


def test_h_table_parity_per_axis():
    """H_iJ(m) with J = (j, k) changes sign under m_a -> -m_a when a appears an odd number of
    times among i, j, k (the entry is a first derivative of the even/odd G_ij)."""
    n, h = (4, 5, 3), 9.0
    H = og.h_table(n, h, W, LAM, MU, RHO)
    for a in range(3):
        ax = 2 + (2 - a)          # array axis of coordinate a in (i, J, z, y, x)
        mirrored = np.flip(np.roll(H, -1, axis=ax), axis=ax)   # index m -> -m mod L
        for i in range(3):
            for J, (j, k) in enumerate(VOIGT):
                s = (-1) ** ((i == a) + (j == a) + (k == a))
                assert np.allclose(mirrored[i, J], s * H[i, J], rtol=0, atol=1e-12 * np.abs(H).max())


@pytest.mark.parametrize("n", [(3, 3, 3), (4, 3, 5)])
def test_h_fft_form_equals_direct_sum(n):
    med = sy.random_medium(n, h=9.0, seed=sum(n) + 70, frac=0.2)
    rng = np.random.default_rng(71)
    u = rng.standard_normal((3,) + med.shape) + 1j * rng.standard_normal((3,) + med.shape)
    want = op.apply_direct_h(u, med, W)
    got = op.FFTOperator(med, W, form="h").apply(u)
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)


def test_h_form_zero_contrast_is_identity():
    med = sy.random_medium((4, 4, 4), h=9.0, seed=72, frac=0.0)
    med.dC[:] = 0.0
    med.drho[:] = 0.0
    u = np.random.default_rng(73).standard_normal((3,) + med.shape) + 0j
    assert np.array_equal(op.FFTOperator(med, W, form="h").apply(u), u)


def _smooth(n, D):
    h = D / (n - 1)
    med = sy.random_medium((n, n, n), h=h, seed=74, frac=0.0)
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    c = D / 2
    bump = np.exp(-((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) / (0.18 * D) ** 2)
    A = np.random.default_rng(75).standard_normal((6, 6))
    A = A + A.T
    med.dC = np.array([A[I, J] * 1e9 * bump for I in range(6) for J in range(I, 6)])
    med.drho = 100.0 * bump
    k = W / 1730.0
    u = np.stack([np.exp(1j * k * X) * np.cos(2 * np.pi * Y / D), np.exp(1j * k * Y),
                  np.exp(1j * k * (X + Z) / np.sqrt(2))])
    return med, u


def test_h_form_agrees_with_difference_form_to_second_order():
    D = 160.0
    diffs = []
    for n in (9, 17):
        med, u = _smooth(n, D)
        fd = op.FFTOperator(med, W).scattered(u)
        hs = op.FFTOperator(med, W, form="h").scattered(u)
        step = (n - 1) // 8
        s = (slice(None),) + (slice(None, None, step),) * 3     # the nodes both grids share
        diffs.append(np.linalg.norm((hs - fd)[s]) / np.linalg.norm(fd[s]))
    assert diffs[1] < 0.05
    assert diffs[1] < 0.35 * diffs[0]      # ~h^2: measured ratio 0.28
