"""Full-size checks at the benchmark's grid (128^3 grf workload) and launch configuration.

The oracle cannot apply the operator at 128^3 in test time, so it evaluates (A u)(x) at a few
sampled nodes by direct summation (``oracle.operator.apply_at_points``) and u0 node by node.
Tolerances: FP64 1e-11 and FP32 2e-5 of max|A u|; the mixed solve must satisfy b - A x = O(tol)
at the samples (relative to max|b|), with A the oracle's FP64 operator.
"""
import numpy as np
import pytest
import torch

import synthetic as sy
from oracle import operator as op, source as osrc
from paper_2301_12836_gb300 import lsm

from gpu_helpers import dev, field, handle, host

pytestmark = pytest.mark.gpu

PTS = [(0, 0, 0), (127, 127, 127), (64, 3, 90), (17, 101, 63), (127, 0, 64)]


@pytest.fixture(scope="module")
def grf128():
    wl = sy.get_workload("grf128_batched")
    return wl, wl.medium()


def _at(a, pts):
    a = a.reshape(3, 128, 128, 128)
    return np.array([a[:, iz, iy, ix] for ix, iy, iz in pts])


def test_apply_128_fp64_and_fp32_sampled(grf128):
    wl, med = grf128
    w = 2 * np.pi * 17.0
    h = handle(med, w, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT)
    u = field(med.shape, 123)
    ud = dev(u).reshape(-1)
    A64 = torch.empty_like(ud)
    lsm.lsm_apply(h, ud, A64)
    u32 = ud.to(torch.complex64)
    A32 = torch.empty_like(u32)
    lsm.lsm_apply_c64(h, u32, A32)
    want = op.apply_at_points(u, med, w, PTS)
    a64 = host(A64)
    scale = np.abs(a64).max()
    assert np.abs(_at(a64, PTS) - want).max() < 1e-11 * scale
    assert np.abs(_at(host(A32).astype(np.complex128), PTS) - want).max() < 2e-5 * scale
    # property at any size: FP32 and FP64 applies agree everywhere to FP32 accuracy
    assert np.linalg.norm(host(A32) - a64) / np.linalg.norm(a64) < 2e-5
    # the mixed solver's double-float residual apply: oracle samples and agreement with FP64
    Adf = torch.empty_like(ud)
    lsm.lsm_apply_df(h, ud, Adf)
    adf = host(Adf)
    assert np.abs(_at(adf, PTS) - want).max() < 1e-11 * scale
    assert np.linalg.norm(adf - a64) / np.linalg.norm(a64) < 1e-11


def test_batched_mixed_solve_128(grf128):
    """8 moment tensors at one frequency in one batched mixed solve, as the bench runs it."""
    wl, med = grf128
    M, xs = wl.sources()
    f = wl.freqs_hz[10]
    w = 2 * np.pi * f
    h = handle(med, w, precision=lsm.LSM_MIXED, tol=1e-6)   # FP64 refinement residual, as the bench
    bs, xsol = [], []
    for j in range(8):
        b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
        assert lsm.lsm_source(h, M[j], xs[j], b) == lsm.LSM_OK
        bs.append(b)
        xsol.append(torch.zeros_like(b))
    code, its, rrs, sts = lsm.lsm_solve_batched([h] * 8, bs, xsol)
    assert code == lsm.LSM_OK and max(rrs) <= 1e-6
    for j in (0, 5):
        bh = host(bs[j])
        u0 = osrc.background_field(med.n, med.h, M[j], xs[j], w, med.lam0, med.mu0, med.rho0)[0]
        assert np.abs(bh.reshape(u0.shape) - u0).max() < 1e-12 * np.abs(u0).max()
        x = host(xsol[j]).reshape(3, 128, 128, 128)
        Ax = op.apply_at_points(x, med, w, PTS[:3])
        assert np.abs(Ax - _at(bh, PTS[:3])).max() < 1e-5 * np.abs(bh).max()


PTS256 = [(255, 130, 128), (77, 200, 12)]   # each costs the oracle ~20 s of direct sums


@pytest.mark.slow
def test_tti256_apply_sampled_and_batched_solve():
    """The largest workload (256^3, TTI layer, dx 5 m): FP64 and FP32 applies at sampled nodes
    against the oracle's direct sums, and the workload's 4 sources at one frequency in one
    batched mixed solve with the residual checked at sampled nodes."""
    wl = sy.get_workload("tti256_batched")
    med = wl.medium()
    n = med.shape
    w = 2 * np.pi * wl.freqs_hz[9]
    h = handle(med, w, precision=lsm.LSM_MIXED, residual=lsm.LSM_RESIDUAL_DFLOAT, tol=1e-6)
    u = field(n, 256)
    ud = dev(u).reshape(-1)
    A64 = torch.empty_like(ud)
    lsm.lsm_apply(h, ud, A64)
    u32 = ud.to(torch.complex64)
    A32 = torch.empty_like(u32)
    lsm.lsm_apply_c64(h, u32, A32)
    del ud, u32
    want = op.apply_at_points(u, med, w, PTS256)
    a64 = host(A64).reshape(3, *n)
    a32 = host(A32).reshape(3, *n).astype(np.complex128)
    del A64, A32
    got64 = np.array([a64[:, iz, iy, ix] for ix, iy, iz in PTS256])
    got32 = np.array([a32[:, iz, iy, ix] for ix, iy, iz in PTS256])
    scale = np.abs(a64).max()
    assert np.abs(got64 - want).max() < 1e-11 * scale
    assert np.abs(got32 - want).max() < 2e-5 * scale
    del a64, a32, u
    M, xs = wl.sources()
    bs = [torch.empty(3 * h.N, dtype=torch.complex128, device="cuda") for _ in M]
    lsm.lsm_source_moments(h, M, xs[0], bs)
    xsol = [torch.zeros_like(b) for b in bs]
    code, its, rrs, sts = lsm.lsm_solve_batched([h] * len(M), bs, xsol)
    assert code == lsm.LSM_OK and max(rrs) <= 1e-6
    x = host(xsol[2]).reshape(3, *n)
    bh = host(bs[2]).reshape(3, *n)
    Ax = op.apply_at_points(x, med, w, PTS256[:1])
    bw = np.array([bh[:, iz, iy, ix] for ix, iy, iz in PTS256[:1]])
    assert np.abs(Ax - bw).max() < 1e-5 * np.abs(bh).max()
