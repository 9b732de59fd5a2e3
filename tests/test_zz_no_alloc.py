"""lsm_apply_static: the FP64 operator apply that makes no device allocation.

It serves callers that cannot call cudaMalloc when they apply the operator: a process whose
device memory was reserved up front by another allocator, or a loop that must not stop on an
out-of-memory error halfway.  Its workspace is the library's static device array, so its result
must equal lsm_apply's and the oracle's, call after call, and a call must not change the
device's free memory.  This file is collected last on purpose: if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import synthetic as sy
from oracle import operator as op
from paper_2301_12836_gb300 import lsm

from gpu_helpers import dev, field, handle, host, rel

pytestmark = pytest.mark.gpu

W = 2 * np.pi * 10.0
STATIC_BYTES = 64 << 20


def _need(n):
    """Bytes of the static array an apply on grid n = (nx, ny, nz) uses: the 256-byte argument
    block and two workspaces of 12 nx ny (nz + 2) complex128 values each."""
    nx, ny, nz = n
    return 256 + 2 * 12 * nx * ny * (nz + 2) * 16


def test_static_apply_equals_lsm_apply_and_the_oracle_on_consecutive_calls():
    med = sy.random_medium((24, 20, 18), h=8.0, seed=31, frac=0.2)
    h = handle(med, W)
    F = op.FFTOperator(med, W)
    for k in range(2):
        u_h = field(med.shape, 40 + k)
        u = dev(u_h).reshape(-1)
        ref = torch.empty_like(u)
        lsm.lsm_apply(h, u, ref)
        out = torch.empty_like(u)
        lsm.lsm_apply_static(h, u, out)
        got = host(out).reshape(u_h.shape)
        assert rel(got, host(ref).reshape(u_h.shape)) < 1e-12
        assert rel(got, F.apply(u_h)) < 1e-12


def test_static_apply_adds_no_device_allocation():
    med = sy.random_medium((16, 12, 20), h=8.0, seed=33, frac=0.2)
    h = handle(med, W)
    u = dev(field(med.shape, 50)).reshape(-1)
    out = torch.empty_like(u)
    lsm.lsm_apply_static(h, u, out)      # first call: the array's address is looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        lsm.lsm_apply_static(h, u, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_apply_accepts_the_largest_grid_and_rejects_the_next():
    # (64, 64, 40) needs 66,060,544 bytes of the 67,108,864; (64, 64, 45) needs 73.9 MB
    fits, too_big = (64, 64, 40), (64, 64, 45)
    assert _need(fits) <= STATIC_BYTES < _need(too_big)
    med = sy.random_medium(fits, h=8.0, seed=34, frac=0.1)
    assert tuple(med.n) == fits
    h = handle(med, W)
    u = dev(field(med.shape, 51)).reshape(-1)
    ref = torch.empty_like(u)
    out = torch.empty_like(u)
    lsm.lsm_apply(h, u, ref)
    lsm.lsm_apply_static(h, u, out)
    assert rel(host(out), host(ref)) < 1e-12
    del h
    med = sy.random_medium(too_big, h=8.0, seed=35, frac=0.1)
    h = handle(med, W)
    u = torch.zeros(3 * h.N, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(u)
    with pytest.raises(lsm.LSMError) as e:
        lsm.lsm_apply_static(h, u, out)
    assert e.value.code == lsm.LSM_ERR_ARG
    assert "static array" in str(e.value)
