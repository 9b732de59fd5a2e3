"""The sampled-H form (LSM_KERNEL_H: Eq. 21 with H of Eq. 9 from the analytic derivative of the
Green's tensor) on the GPU against the oracle's FFT evaluation of the same form.

Tolerances: FP64 apply 1e-12 relative L2 (rounding of two 3-D FFT chains); FP32 apply 1e-5;
solves as in the difference form (FP64 to 1e-11 -> 1e-9, mixed to 1e-8 -> 1e-6).
"""
import numpy as np
import pytest
import torch

import synthetic as sy
from oracle import operator as op, solver as osv, source as osrc
from paper_2301_12836_gb300 import lsm

from gpu_helpers import dev, field, handle, host, rel

pytestmark = pytest.mark.gpu

W = 2 * np.pi * 9.0
H = lsm.LSM_KERNEL_H


# four-step lengths 16/32/64 on every axis, a generic mixed-radix one (2n = 24, 50, 10) and
# ragged tails
GRIDS = [(5, 3, 4), (16, 16, 16), (12, 25, 9), (8, 32, 16)]


@pytest.mark.parametrize("n", GRIDS)
@pytest.mark.parametrize("mode,green", [("exact", lsm.LSM_GREEN_EXACT), ("paper", lsm.LSM_GREEN_PAPER)])
def test_apply_h_fp64_parity(n, mode, green):
    med = sy.random_medium(n, h=8.0, seed=sum(n) + 80, frac=0.2)
    h = handle(med, W, green=green, kernel=H)
    u = field(med.shape, 81)
    Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply(h, dev(u).reshape(-1), Au)
    want = op.FFTOperator(med, W, mode=mode, form="h").apply(u)
    assert rel(host(Au).reshape(want.shape), want) < 1e-12
    # and it is a different operator from the difference form
    assert rel(op.FFTOperator(med, W, mode=mode).apply(u), want) > 1e-6


@pytest.mark.parametrize("precision", [lsm.LSM_FP64, lsm.LSM_MIXED])
def test_apply_h_with_taper_and_paper_green(precision):
    """Options combine: the sampled-H form with the paper's Green's tensor (A.4 + A.5 and its
    derivatives A.6-A.11) and an absorbing layer of 3 nodes (Eq. 25)."""
    med = sy.random_medium((15, 12, 10), h=9.0, seed=87, frac=0.2)
    h = handle(med, W, precision=precision, green=lsm.LSM_GREEN_PAPER, kernel=H, taper=3)
    want_op = op.FFTOperator(op.tapered(med, 3), W, mode="paper", form="h")
    if precision == lsm.LSM_FP64:
        u = field(med.shape, 88)
        Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
        lsm.lsm_apply(h, dev(u).reshape(-1), Au)
        want = want_op.apply(u)
        assert rel(host(Au).reshape(want.shape), want) < 1e-12
    else:
        u = field(med.shape, 88, np.complex64)
        Au = torch.empty(3 * h.N, dtype=torch.complex64, device="cuda")
        lsm.lsm_apply_c64(h, dev(u).reshape(-1), Au)
        want = want_op.apply(u.astype(np.complex128))
        assert rel(host(Au).reshape(want.shape).astype(np.complex128), want) < 1e-5


@pytest.mark.parametrize("n", [(16, 16, 16), (12, 25, 9)])
def test_apply_h_fp32_parity(n):
    med = sy.random_medium(n, h=8.0, seed=sum(n) + 82, frac=0.2)
    h = handle(med, W, precision=lsm.LSM_MIXED, kernel=H)
    u = field(med.shape, 83, np.complex64)
    Au = torch.empty(3 * h.N, dtype=torch.complex64, device="cuda")
    lsm.lsm_apply_c64(h, dev(u).reshape(-1), Au)
    want = op.FFTOperator(med, W, form="h").apply(u.astype(np.complex128))
    assert rel(host(Au).reshape(want.shape).astype(np.complex128), want) < 1e-5


@pytest.mark.parametrize("precision,tol,bar", [(lsm.LSM_FP64, 1e-11, 1e-9), (lsm.LSM_MIXED, 1e-8, 1e-6)])
def test_solve_h_batched(precision, tol, bar):
    """Two frequencies x one source each, batched, in the sampled-H form, against the oracle."""
    med = sy.random_medium((10, 12, 9), h=10.0, seed=84, frac=0.1)
    ws = [2 * np.pi * 6.0, 2 * np.pi * 13.0]
    h0 = handle(med, ws[0], precision=precision, tol=tol, kernel=H)
    h1 = lsm.lsm_create_shared(h0, ws[1])
    xs_ = np.array([44.0, 51.0, 37.0])
    bs, xs, want = [], [], []
    for hh, w in ((h0, ws[0]), (h1, ws[1])):
        b = torch.empty(3 * hh.N, dtype=torch.complex128, device="cuda")
        lsm.lsm_source(hh, sy.double_couple_13(), xs_, b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
        u0, _ = osrc.background_field(med.n, med.h, sy.double_couple_13(), xs_, w, med.lam0, med.mu0, med.rho0)
        xo, *_ = osv.bicgstab(op.FFTOperator(med, w, form="h").apply, u0, tol=1e-13, maxit=400)
        want.append(xo)
    code, its, rrs, sts = lsm.lsm_solve_batched([h0, h1], bs, xs)
    assert code == lsm.LSM_OK and all(s == 0 for s in sts)
    for x, xo, rr in zip(xs, want, rrs):
        assert rr <= tol
        assert rel(host(x).reshape(xo.shape), xo) < bar


def test_h_form_rejects_adjoint_calls():
    med = sy.random_medium((6, 5, 4), h=10.0, seed=85, frac=0.1)
    h = handle(med, W, kernel=H)
    v = dev(field(med.shape, 86)).reshape(-1)
    out = torch.empty_like(v)
    for call in (lambda: lsm.lsm_adjoint(h, v, out), lambda: lsm.lsm_solve_adjoint(h, v, out),
                 lambda: lsm.lsm_apply_static(h, v, out)):
        with pytest.raises(lsm.LSMError) as e:
            call()
        assert e.value.code == lsm.LSM_ERR_ARG
    gC = torch.zeros(21 * h.N, dtype=torch.float64, device="cuda")
    gr = torch.zeros(h.N, dtype=torch.float64, device="cuda")
    with pytest.raises(lsm.LSMError):
        lsm.lsm_gradient(h, v, v, gC, gr)
