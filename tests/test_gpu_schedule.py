"""FFT schedule variants and the tuner: every variant of every stage computes the same operator
(parity with the oracle at the apply tolerances: FP64 1e-12, FP32 1e-5), and a tuned schedule
solves to the same solution."""
import numpy as np
import pytest
import torch

import synthetic as sy
from oracle import operator as op
from paper_2301_12836_gb300 import lsm

from gpu_helpers import dev, field, handle, host, rel

pytestmark = pytest.mark.gpu

W = 2 * np.pi * 9.0
VARIANTS = [[0, 0, 0, 0, 0, 0], [0, 1, 1, 1, 1, 1], [0, 2, 2, 2, 2, 2], [0, 0, 0, 3, 0, 0], [0, 1, 0, 2, 1, 0],
            [1, 0, 0, 0, 0, 0], [1, 1, 1, 1, 1, 1]]


@pytest.mark.parametrize("n", [(16, 16, 16), (12, 25, 9), (8, 32, 16)])
@pytest.mark.parametrize("v", VARIANTS)
def test_every_schedule_variant_gives_the_operator(n, v):
    med = sy.random_medium(n, h=8.0, seed=sum(n) + 90, frac=0.2)
    want = op.FFTOperator(med, W).apply(field(med.shape, 91))
    h64 = handle(med, W)
    lsm.lsm_set_schedule(h64, lsm.LSM_FP64, v)
    assert lsm.lsm_get_schedule(h64, lsm.LSM_FP64) == v
    Au = torch.empty(3 * h64.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply(h64, dev(field(med.shape, 91)).reshape(-1), Au)
    assert rel(host(Au).reshape(want.shape), want) < 1e-12
    h32 = handle(med, W, precision=lsm.LSM_MIXED)
    lsm.lsm_set_schedule(h32, lsm.LSM_MIXED, v)
    u32 = field(med.shape, 91).astype(np.complex64)
    Au32 = torch.empty(3 * h32.N, dtype=torch.complex64, device="cuda")
    lsm.lsm_apply_c64(h32, dev(u32).reshape(-1), Au32)
    want32 = op.FFTOperator(med, W).apply(u32.astype(np.complex128))
    assert rel(host(Au32).reshape(want.shape).astype(np.complex128), want32) < 1e-5


@pytest.mark.parametrize("n", [(16, 16, 16), (36, 9, 5), (2, 2, 2)])
@pytest.mark.parametrize("precision", [lsm.LSM_FP64, lsm.LSM_MIXED])
def test_fused_contraction_is_bitwise_the_separate_kernels(n, precision):
    """Stage-0 variant 1 (contraction and divergence fused, z-marching tiles with halos) does the
    arithmetic of the separate stress and divergence kernels in the same order: bitwise equal."""
    med = sy.random_medium(n, h=8.0, seed=sum(n) + 94, frac=0.2)
    h = handle(med, W, precision=precision)
    ctype = torch.complex128 if precision == lsm.LSM_FP64 else torch.complex64
    u = dev(field(med.shape, 95)).reshape(-1).to(ctype)
    outs = []
    for v0 in (0, 1):
        lsm.lsm_set_schedule(h, precision, [v0, 0, 0, 0, 0, 0])
        Au = torch.empty_like(u)
        (lsm.lsm_apply if precision == lsm.LSM_FP64 else lsm.lsm_apply_c64)(h, u, Au)
        outs.append(Au)
    assert torch.equal(outs[0], outs[1])


def test_bad_schedules_rejected():
    med = sy.random_medium((6, 6, 6), h=8.0, seed=92)
    h = handle(med, W)
    for v in ([2, 0, 0, 0, 0, 0], [0, 3, 0, 0, 0, 0], [0, 0, 0, 4, 0, 0], [0, -1, 0, 0, 0, 0]):
        with pytest.raises(lsm.LSMError):
            lsm.lsm_set_schedule(h, lsm.LSM_FP64, v)


def test_autotune_then_solve():
    med = sy.random_medium((32, 32, 32), h=10.0, seed=93, frac=0.05)
    h = handle(med, W, precision=lsm.LSM_MIXED, tol=1e-7)
    b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_source(h, sy.explosion(), [151.0, 157.0, 149.0], b)
    x0 = torch.zeros_like(b)
    code, _, rr0 = lsm.lsm_solve(h, b, x0)
    assert code == lsm.LSM_OK and rr0 <= 1e-7
    v64, v32 = lsm.lsm_autotune(h, 3, 2)
    assert v64[0] == 0 and v32[0] == 0 and all(0 <= v <= 3 for v in v64 + v32)
    assert lsm.lsm_get_schedule(h, lsm.LSM_FP64) == v64 and lsm.lsm_get_schedule(h, lsm.LSM_MIXED) == v32
    x1 = torch.zeros_like(b)
    code, _, rr1 = lsm.lsm_solve(h, b, x1)
    assert code == lsm.LSM_OK and rr1 <= 1e-7
    assert rel(host(x1), host(x0)) < 1e-6
