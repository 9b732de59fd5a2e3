"""lsm_apply_static: the FP64 operator apply that makes no device allocation.

It serves callers that cannot call cudaMalloc when they apply the operator (a stream being
captured into a CUDA graph, memory reserved up front by another allocator, loops that must
not fail on out-of-memory).  Its workspace is the library's static device array, so its
result must equal lsm_apply's, call after call.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synthetic as sy
from paper_2301_12836_gb300 import lsm

from gpu_helpers import dev, field, handle, host, rel

pytestmark = pytest.mark.gpu

W = 2 * np.pi * 10.0


def test_static_apply_equals_lsm_apply_on_consecutive_calls():
    med = sy.random_medium((24, 20, 18), h=8.0, seed=31, frac=0.2)
    h = handle(med, W)
    for k in range(2):
        u = dev(field(med.shape, 40 + k)).reshape(-1)
        ref = torch.empty_like(u)
        lsm.lsm_apply(h, u, ref)
        out = torch.empty_like(u)
        lsm.lsm_apply_static(h, u, out)
        assert rel(host(out), host(ref)) < 1e-12


def test_static_apply_rejects_a_grid_beyond_the_array():
    med = sy.random_medium((64, 64, 64), h=8.0, seed=32, frac=0.1)
    h = handle(med, W)
    u = torch.zeros(3 * h.N, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(u)
    with pytest.raises(lsm.LSMError) as e:
        lsm.lsm_apply_static(h, u, out)
    assert e.value.code == lsm.LSM_ERR_ARG
    assert "static array" in str(e.value)
