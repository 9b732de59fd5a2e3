"""BiCGSTAB inner products summed in the operator epilogue (lsm_opts.fused_dots).

With fused_dots = 1 the apply that writes v = A p also sums <r^, v> and the one that writes
t = A s sums <t, s> and <t, t> (van der Vorst's BiCGSTAB, the alpha and omega steps of the
iteration used for Eq. 22) in the FP32 iterations of mixed solves, on grids whose x side doubles to
16, 64 or 256.  These tests solve the same systems with the epilogue sums and with the separate
vector kernels, check both against the oracle's BiCGSTAB, and check that the fused path is
deterministic.
"""
import numpy as np
import pytest
import torch

import synthetic as sy
from oracle import operator as op, solver as osv, source as osrc
from paper_2301_12836_gb300 import lsm
from tests.gpu_helpers import handle, host, rel

pytestmark = pytest.mark.gpu

# x sides 8 and 32: the padded x length is 16 or 64, where the epilogue is the warp-per-line pass
GRIDS = [(8, 6, 10), (32, 12, 10)]


def _systems(med, ws):
    srcs = [(sy.explosion(), np.array([0.37, 0.41, 0.52])), (sy.double_couple_13(), np.array([0.63, 0.55, 0.45]))]
    ext = np.array(med.n, dtype=float) * med.h
    out = []
    for w in ws:
        for M, frac in srcs:
            out.append((w, M, frac * ext))
    return out


def _solve(med, systems, precision, tol, fused, graph=1):
    h0 = handle(med, systems[0][0], precision=precision, tol=tol, fused_dots=fused, graph=graph)
    shared = {systems[0][0]: h0}
    hs, bs, xs = [], [], []
    for w, M, s in systems:
        if w not in shared:
            shared[w] = lsm.lsm_create_shared(h0, w)
        hh = shared[w]
        b = torch.empty(3 * hh.N, dtype=torch.complex128, device="cuda")
        lsm.lsm_source(hh, M, s, b)
        hs.append(hh)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    n0 = lsm.lsm_launch_count(h0)
    code, its, rrs, sts = lsm.lsm_solve_batched(hs, bs, xs)
    launches = lsm.lsm_launch_count(h0) - n0
    return code, its, rrs, sts, [host(x) for x in xs], launches, (h0, shared)


@pytest.mark.parametrize("n", GRIDS)
def test_fused_dots_match_vector_kernels_and_oracle(n):
    """Mixed solves (FP32 iterations, the ones that fuse) with and without the epilogue sums."""
    tol, bar = 1e-8, 1e-6
    med = sy.random_medium(n, h=10.0, seed=5, frac=0.1)
    systems = _systems(med, [2 * np.pi * 7.0, 2 * np.pi * 13.0])
    res = {f: _solve(med, systems, lsm.LSM_MIXED, tol, f) for f in (0, 1)}
    for f in (0, 1):
        code, its, rrs, sts, xs, _, _ = res[f]
        assert code == lsm.LSM_OK and all(s == 0 for s in sts) and all(r <= tol for r in rrs)
    for k, (w, M, s) in enumerate(systems):
        u0, _ = osrc.background_field(med.n, med.h, M, s, w, med.lam0, med.mu0, med.rho0)
        xo, *_ = osv.bicgstab(op.FFTOperator(med, w).apply, u0, tol=1e-13, maxit=600)
        for f in (0, 1):
            assert rel(res[f][4][k].reshape(xo.shape), xo) < bar
        # the two summation orders differ only by rounding: the same inner iteration counts within
        # one per inner solve (at most the refinement steps taken)
        assert abs(res[0][1][k] - res[1][1][k]) <= 4


def test_fused_dots_leave_fp64_solves_unchanged():
    """FP64 iterations keep the vector kernels whatever fused_dots says: bitwise the same solves
    and the same launches."""
    med = sy.random_medium((8, 6, 10), h=10.0, seed=5, frac=0.1)
    systems = _systems(med, [2 * np.pi * 7.0])
    res = {f: _solve(med, systems, lsm.LSM_FP64, 1e-11, f) for f in (0, 1)}
    assert res[0][0] == res[1][0] == lsm.LSM_OK
    assert all(np.array_equal(a, b) for a, b in zip(res[0][4], res[1][4]))
    assert res[0][1] == res[1][1] and res[0][5] == res[1][5]


def test_fused_dots_graph_replay_is_bitwise_eager():
    """The epilogue sums reduce in block order like the vector kernels: replaying the captured
    iterations gives bitwise the eager iterates, and a second solve repeats them."""
    med = sy.random_medium((8, 10, 9), h=10.0, seed=17, frac=0.1)
    systems = _systems(med, [2 * np.pi * 9.0])
    out = {}
    for graph in (0, 1):
        runs = [_solve(med, systems, lsm.LSM_MIXED, 1e-8, 1, graph=graph) for _ in range(2)]
        for r in runs:
            assert r[0] == lsm.LSM_OK
        assert all(np.array_equal(a, b) for a, b in zip(runs[0][4], runs[1][4])) and runs[0][1] == runs[1][1]
        out[graph] = runs[0]
    assert all(np.array_equal(a, b) for a, b in zip(out[0][4], out[1][4]))
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]


def test_fused_dots_zero_rhs_and_unequal_stops():
    """A zero right-hand side (no iteration runs for it) and systems that stop at different
    iterations share the batch: the stopped systems' epilogue blocks return before their sums,
    and the others still converge."""
    med = sy.random_medium((8, 6, 10), h=10.0, seed=23, frac=0.3)
    w = 2 * np.pi * 30.0
    tol = 1e-8
    h = handle(med, w, precision=lsm.LSM_MIXED, tol=tol, fused_dots=1)
    h2 = lsm.lsm_create_shared(h, 2 * np.pi * 1.0)   # low frequency: fewer iterations (oracle: 6 vs 9)
    b0 = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    s = np.array(med.n, dtype=float) * med.h * 0.45
    lsm.lsm_source(h, sy.explosion(), s, b0)
    b1 = torch.zeros_like(b0)
    b2 = torch.empty_like(b0)
    lsm.lsm_source(h2, sy.explosion(), s, b2)
    # a nonzero initial guess of the solution's scale for the first system (the Born field b)
    xs = [0.5 * b0, torch.full_like(b0, 2.0), torch.zeros_like(b0)]
    code, its, rrs, sts = lsm.lsm_solve_batched([h, h, h2], [b0, b1, b2], xs)
    assert code == lsm.LSM_OK and list(sts) == [0, 0, 0] and all(r <= tol for r in rrs)
    assert torch.count_nonzero(xs[1]).item() == 0
    assert its[2] <= its[0]   # inner iterations summed over the refinement steps
    for x, b, ww in ((xs[0], b0, w), (xs[2], b2, 2 * np.pi * 1.0)):
        u0 = host(b).reshape((3,) + tuple(med.n[::-1]))
        assert osv.relres(op.FFTOperator(med, ww).apply, u0, host(x).reshape(u0.shape)) < 10 * tol
