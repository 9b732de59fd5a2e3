"""The operator in double-float arithmetic (lsm_apply_df) and the mixed solver's double-float
refinement residual, against the FP64 oracle.

Tolerance of the apply: relative L2 1e-11.  Each double-float operation rounds with a normwise
error of a few u^2 (u = 2^-24, u^2 = 3.6e-15) times the magnitude of its operands; an entry of
A u passes through about 80 dependent operations (three forward and three inverse radix passes of
log2 L stages each, the stencils, the 21-term contraction and the 6-term Green products), so the
error stays near 80 * 3 * 3.6e-15 ~ 1e-12.  1e-11 leaves a factor of ten and is still 10^4 below
the FP32 apply's error, the gap the refinement residual needs.
"""
import numpy as np
import pytest
import torch

import synthetic as sy
from oracle import operator as op, solver as osv, source as osrc
from paper_2301_12836_gb300 import lsm

from gpu_helpers import dev, field, handle, host, rel

pytestmark = pytest.mark.gpu

W = 2 * np.pi * 10.0


# (128, ., .) etc. run the compile-time 16 x 16 engine of the double-float path along that axis,
# with ragged tiles on the short axes; the others run the generic engine on every axis
@pytest.mark.parametrize("n", [(20, 18, 15), (12, 10, 8), (128, 6, 5), (5, 128, 6), (6, 5, 128), (128, 9, 128)])
def test_apply_df_parity(n):
    med = sy.random_medium(n, h=8.0, seed=sum(n) + 1, frac=0.2)
    h = handle(med, W, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT)
    u = field(med.shape, 11)
    Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply_df(h, dev(u).reshape(-1), Au)
    want = op.FFTOperator(med, W).apply(u)
    got = host(Au).reshape(u.shape)
    assert rel(got, want) < 1e-11
    # the scattered part alone (u - A u), where the arithmetic happens
    assert rel(u - got, u - want) < 1e-10


def test_apply_df_green_paper_and_taper():
    med = sy.random_medium((16, 12, 10), h=8.0, seed=71, frac=0.2)
    h = handle(med, W, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT, green=lsm.LSM_GREEN_PAPER, taper=3)
    u = field(med.shape, 12)
    Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply_df(h, dev(u).reshape(-1), Au)
    want = op.FFTOperator(op.tapered(med, 3), W, "paper").apply(u)
    assert rel(host(Au).reshape(u.shape), want) < 1e-11


@pytest.mark.parametrize("n", [(16, 12, 10), (128, 6, 5)])
@pytest.mark.parametrize("mode,green", [("exact", lsm.LSM_GREEN_EXACT), ("paper", lsm.LSM_GREEN_PAPER)])
def test_apply_df_hform_parity(n, mode, green):
    """The sampled-H form (Eq. 21 with the analytic H) in double-float arithmetic."""
    med = sy.random_medium(n, h=8.0, seed=sum(n) + 5, frac=0.2)
    h = handle(med, W, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT, green=green, kernel=lsm.LSM_KERNEL_H)
    u = field(med.shape, 14)
    Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply_df(h, dev(u).reshape(-1), Au)
    want = op.FFTOperator(med, W, mode=mode, form="h").apply(u)
    got = host(Au).reshape(u.shape)
    assert rel(got, want) < 1e-11
    assert rel(u - got, u - want) < 1e-10


def test_mixed_solve_hform_pair_residual():
    """A batched mixed solve of the sampled-H form with the double-float residual against the
    oracle's solution of the same form."""
    med = sy.random_medium((12, 10, 9), h=10.0, seed=75, frac=0.1)
    w = 2 * np.pi * 9.0
    h = handle(med, w, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT, tol=1e-8, kernel=lsm.LSM_KERNEL_H)
    srcs = [(sy.explosion(), np.array([44.0, 41.0, 37.0])), (sy.double_couple_12(), np.array([31.0, 52.0, 45.0]))]
    bs, xs_, want = [], [], []
    F = op.FFTOperator(med, w, form="h")
    for M, s in srcs:
        b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
        lsm.lsm_source(h, M, s, b)
        bs.append(b)
        xs_.append(torch.zeros_like(b))
        u0 = host(b).reshape((3,) + med.shape)
        xo, *_ = osv.bicgstab(F.apply, u0, tol=1e-12, maxit=400)
        want.append(xo)
    code, its, rrs, sts = lsm.lsm_solve_batched([h] * 2, bs, xs_)
    assert code == lsm.LSM_OK
    for x, xo, rr, b in zip(xs_, want, rrs, bs):
        assert rr <= 1e-8
        assert rel(host(x).reshape(xo.shape), xo) < 1e-6
        u0 = host(b).reshape(xo.shape)
        assert abs(osv.relres(F.apply, u0, host(x).reshape(xo.shape)) - rr) < 1e-9


def test_apply_df_rejects_other_handles():
    med = sy.random_medium((8, 8, 8), h=10.0, seed=72, frac=0.1)
    u = dev(field(med.shape, 13)).reshape(-1)
    Au = torch.empty_like(u)
    for kw in (dict(precision=lsm.LSM_FP64), dict(precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_FP64)):
        h = handle(med, W, **kw)
        with pytest.raises(lsm.LSMError):
            lsm.lsm_apply_df(h, u, Au)


@pytest.mark.parametrize("scale", [1.0, 1e-28, 1e28])
def test_mixed_solve_pair_residual(scale):
    """Mixed solves with the double-float residual: the same answer as with the FP64 residual and as
    the oracle, also for right-hand sides far outside FP32's comfortable range (the iterate is
    scaled by a power of two before the pair apply); the reported residual is the true one."""
    med = sy.random_medium((15, 12, 10), h=10.0, seed=73, frac=0.15)
    w = 2 * np.pi * 8.0
    xs = np.array([61.0, 52.0, 47.0])
    M = sy.double_couple_13() * scale
    sols = {}
    for res in (lsm.LSM_RESIDUAL_DFLOAT, lsm.LSM_RESIDUAL_FP64):
        h = handle(med, w, precision=lsm.LSM_MIXED, tol=1e-8, residual=res)
        b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
        lsm.lsm_source(h, M, xs, b)
        x = torch.zeros_like(b)
        code, it, rr = lsm.lsm_solve(h, b, x)
        assert code == lsm.LSM_OK and rr <= 1e-8
        sols[res] = (host(x), rr)
    u0, _ = osrc.background_field(med.n, med.h, M, xs, w, med.lam0, med.mu0, med.rho0)
    F = op.FFTOperator(med, w)
    xo, *_ = osv.bicgstab(F.apply, u0, tol=1e-12, maxit=400)
    for res, (x, rr) in sols.items():
        assert rel(x.reshape(u0.shape), xo) < 1e-6
        assert abs(osv.relres(F.apply, u0, x.reshape(u0.shape)) - rr) < 1e-9


def test_mixed_solve_pair_residual_nonzero_guess():
    """A nonzero initial iterate enters the first pair apply scaled by its own norm."""
    med = sy.random_medium((10, 9, 8), h=10.0, seed=74, frac=0.15)
    w = 2 * np.pi * 7.0
    h = handle(med, w, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT, tol=1e-9)
    b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_source(h, sy.explosion(), [41.0, 33.0, 29.0], b)
    x = b.clone() * 1e-3
    code, it, rr = lsm.lsm_solve(h, b, x)
    assert code == lsm.LSM_OK and rr <= 1e-9
    u0 = host(b).reshape((3,) + med.shape)
    assert abs(osv.relres(op.FFTOperator(med, w).apply, u0, host(x).reshape(u0.shape)) - rr) < 1e-10
