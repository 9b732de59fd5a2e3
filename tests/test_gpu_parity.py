"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 unless stated):
* FP64 apply / adjoint / source: 1e-12.  Both sides evaluate the same sums in
  FP64; FFT rounding grows like u log2(P) ~ 1e-15 * 20, well below 1e-12.
* FP32 apply: 1e-5.  FP32 FFTs and contraction carry ~6e-8 * log2(P) relative
  error on the scattered part, a fraction of the field.
* FP64 solve: 1e-10 with both sides solved to relres 1e-12 (cond(A) is O(10)).
* mixed solve: 1e-6 with the mixed solve taken to relres 1e-8.
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


def _oracle_apply(med, omega, u, mode="exact"):
    return op.FFTOperator(med, omega, mode).apply(u)


@pytest.mark.parametrize("mode,green", [("exact", lsm.LSM_GREEN_EXACT), ("paper", lsm.LSM_GREEN_PAPER)])
def test_source_parity(mode, green):
    med = sy.random_medium((9, 5, 6), h=10.0, seed=21)
    h = handle(med, W, green=green)
    xs = np.array([41.3, 27.9, 55.2])
    M = np.array([0.3, -1.2, 0.7, 0.25, -0.4, 0.9])
    u0 = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    code = lsm.lsm_source(h, M, xs, u0)
    assert code == lsm.LSM_OK
    want, hit = osrc.background_field(med.n, med.h, M, xs, W, med.lam0, med.mu0, med.rho0, mode)
    assert not hit
    assert rel(host(u0).reshape(want.shape), want) < 1e-12


@pytest.mark.parametrize("mode,green", [("exact", lsm.LSM_GREEN_EXACT), ("paper", lsm.LSM_GREEN_PAPER)])
def test_source_moments_parity(mode, green):
    """Ten moment tensors at one position (two launches of up to eight): each field matches the
    oracle and is bitwise the field lsm_source gives for that tensor alone."""
    med = sy.random_medium((12, 10, 9), h=10.0, seed=23)
    h = handle(med, W, green=green)
    xs = np.array([53.1, 41.7, 38.4])
    Ms = sy.random_moment_tensors(10, np.random.default_rng(24))
    outs = [torch.empty(3 * h.N, dtype=torch.complex128, device="cuda") for _ in Ms]
    assert lsm.lsm_source_moments(h, Ms, xs, outs) == lsm.LSM_OK
    for M, u0 in zip(Ms, outs):
        want, _ = osrc.background_field(med.n, med.h, M, xs, W, med.lam0, med.mu0, med.rho0, mode)
        assert rel(host(u0).reshape(want.shape), want) < 1e-12
        one = torch.empty_like(u0)
        lsm.lsm_source(h, M, xs, one)
        assert torch.equal(one, u0)


def test_source_moments_on_node_and_bad_arguments():
    med = sy.random_medium((6, 6, 6), h=10.0, seed=22)
    h = handle(med, W)
    outs = [torch.empty(3 * h.N, dtype=torch.complex128, device="cuda") for _ in range(2)]
    Ms = [sy.explosion(), sy.double_couple_12()]
    assert lsm.lsm_source_moments(h, Ms, [20.0, 30.0, 40.0], outs) == lsm.LSM_WARN_SOURCE_ON_NODE
    for u0 in outs:
        assert np.all(host(u0).reshape(3, 6, 6, 6)[:, 4, 3, 2] == 0)
    with pytest.raises(lsm.LSMError):
        lsm.lsm_source_moments(h, [[np.nan] * 6], [1.0, 2.0, 3.0], outs[:1])
    with pytest.raises(lsm.LSMError):
        lsm.lsm_source_moments(h, [], [1.0, 2.0, 3.0], [])


@pytest.mark.parametrize("n", [1, 4097, 3 * 1000003])
def test_fp32_inner_products_are_fp64_accurate(n):
    """The FP32 solver's inner products (exact products, compensated partial sums, FP64 totals)
    against the correctly rounded sum of the exact products (math.fsum of FP64 products of the
    FP32 values, which are exact): error <= 1e-11 of sum |terms|, including a sum that cancels."""
    import math
    med = sy.random_medium((4, 4, 4), h=10.0, seed=25)
    h = handle(med, W, precision=lsm.LSM_MIXED)
    rng = np.random.default_rng(n)
    a = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.exp(3 * rng.standard_normal(n))).astype(np.complex64)
    b = ((rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.exp(3 * rng.standard_normal(n))).astype(np.complex64)
    for bb in (b, (1j * a).astype(np.complex64)):        # i a: the real part cancels exactly
        ax, ay = a.real.astype(np.float64), a.imag.astype(np.float64)
        bx, by = bb.real.astype(np.float64), bb.imag.astype(np.float64)
        re_terms = np.concatenate([ax * bx, ay * by])
        im_terms = np.concatenate([ax * by, -ay * bx])
        got = lsm.lsm_dot_c64(h, dev(a), dev(bb))
        for g, terms in ((got.real, re_terms), (got.imag, im_terms)):
            exact = math.fsum(terms)
            assert abs(g - exact) <= 1e-11 * np.abs(terms).sum() + 1e-300, (g, exact)


def test_source_on_node_flag():
    med = sy.random_medium((6, 6, 6), h=10.0, seed=22)
    h = handle(med, W)
    u0 = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    code = lsm.lsm_source(h, sy.explosion(), [20.0, 30.0, 40.0], u0)
    assert code == lsm.LSM_WARN_SOURCE_ON_NODE
    got = host(u0).reshape(3, 6, 6, 6)
    assert np.all(got[:, 4, 3, 2] == 0)
    want, hit = osrc.background_field(med.n, med.h, sy.explosion(), np.array([20.0, 30.0, 40.0]), W,
                                      med.lam0, med.mu0, med.rho0)
    assert hit and rel(got, want) < 1e-12


# grids spanning several tiles in every pass, ragged tails, odd and non-cubic sizes, minimum size
# (8, 32, 16) and (64, 8, 12) run every axis through a different FFT engine (four-step 16/64/32,
# four-step 128 / 16 and generic 24)
GRIDS = [(2, 2, 2), (5, 3, 4), (20, 18, 15), (16, 16, 16), (12, 25, 9), (8, 32, 16), (64, 8, 12), (32, 32, 32), (8, 8, 8)]


@pytest.mark.parametrize("n", GRIDS)
@pytest.mark.parametrize("mode,green", [("exact", lsm.LSM_GREEN_EXACT), ("paper", lsm.LSM_GREEN_PAPER)])
def test_apply_fp64_parity(n, mode, green):
    med = sy.random_medium(n, h=8.0, seed=sum(n), frac=0.2)
    h = handle(med, W, green=green)
    u = field(med.shape, 1)
    Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply(h, dev(u).reshape(-1), Au)
    want = _oracle_apply(med, W, u, mode)
    assert rel(host(Au).reshape(u.shape), want) < 1e-12
    assert rel(u, want) > 1e-3  # the scattered part is resolved


@pytest.mark.parametrize("n", [(20, 18, 15), (16, 16, 16), (8, 32, 16), (64, 8, 12), (32, 32, 32), (8, 8, 8)])
def test_apply_fp32_parity(n):
    med = sy.random_medium(n, h=8.0, seed=3, frac=0.2)
    h = handle(med, W, precision=lsm.LSM_MIXED)
    u = field(med.shape, 2)
    Au = torch.empty(3 * h.N, dtype=torch.complex64, device="cuda")
    lsm.lsm_apply_c64(h, dev(u, torch.complex64).reshape(-1), Au)
    want = _oracle_apply(med, W, u)
    assert rel(host(Au).reshape(u.shape).astype(np.complex128), want) < 1e-5


@pytest.mark.parametrize("n", [(5, 3, 4), (20, 18, 15)])
def test_adjoint_parity(n):
    med = sy.random_medium(n, h=8.0, seed=5, frac=0.2)
    h = handle(med, W)
    w = field(med.shape, 3)
    out = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_adjoint(h, dev(w).reshape(-1), out)
    want = op.FFTOperator(med, W).adjoint(w)
    assert rel(host(out).reshape(w.shape), want) < 1e-12
    # dot-product test through the GPU alone: <A v, w> = <v, A^H w>
    v = field(med.shape, 4)
    Av = torch.empty_like(out)
    lsm.lsm_apply(h, dev(v).reshape(-1), Av)
    lhs = np.vdot(w.reshape(-1), host(Av))
    rhs = np.vdot(host(out), v.reshape(-1))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_zero_contrast_is_identity_bitwise():
    med = sy.random_medium((12, 10, 9), seed=6)
    med.dC[:] = 0
    med.drho[:] = 0
    h = handle(med, W, precision=lsm.LSM_MIXED)
    u = dev(field(med.shape, 5)).reshape(-1)
    Au = torch.empty_like(u)
    lsm.lsm_apply(h, u, Au)
    assert torch.equal(Au, u)
    u32 = u.to(torch.complex64)
    A32 = torch.empty_like(u32)
    lsm.lsm_apply_c64(h, u32, A32)
    assert torch.equal(A32, u32)


def test_solve_fp64_inclusion16():
    """16^3 VTI cube inclusion, explosion at the centre, 10 Hz, FP64 solve vs the oracle's BiCGSTAB."""
    wl = sy.get_workload("inclusion16_fp64")
    med = wl.medium()
    M, xs = wl.sources()
    w = 2 * np.pi * wl.freqs_hz[0]
    h = handle(med, w, tol=1e-12)
    b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    assert lsm.lsm_source(h, M[0], xs[0], b) == lsm.LSM_OK
    x = torch.zeros_like(b)
    code, it, rr = lsm.lsm_solve(h, b, x)
    assert code == lsm.LSM_OK and rr <= 1e-12
    u0, _ = osrc.background_field(med.n, med.h, M[0], xs[0], w, med.lam0, med.mu0, med.rho0)
    xo, ito, rro, sto, _ = osv.bicgstab(op.FFTOperator(med, w).apply, u0, tol=1e-12, maxit=200)
    assert sto == 0
    assert rel(host(x).reshape(u0.shape), xo) < 1e-10
    assert abs(it - ito) <= 1


def test_solve_mixed_layers():
    """Three VTI layers (the 64^3 workload's medium at 24^3), strike-slip source, mixed solve to 1e-8."""
    med = sy.layered_vti_medium(24, 10.0)
    w = 2 * np.pi * 15.0
    h = handle(med, w, precision=lsm.LSM_MIXED, tol=1e-8)
    xs = np.array([115.0, 115.0, 120.0])
    b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_source(h, sy.double_couple_12(), xs, b)
    x = torch.zeros_like(b)
    code, it, rr = lsm.lsm_solve(h, b, x)
    assert code == lsm.LSM_OK and rr <= 1e-8
    u0, _ = osrc.background_field(med.n, med.h, sy.double_couple_12(), xs, w, med.lam0, med.mu0, med.rho0)
    F = op.FFTOperator(med, w)
    xo, *_ = osv.bicgstab(F.apply, u0, tol=1e-12, maxit=400)
    assert rel(host(x).reshape(u0.shape), xo) < 1e-6
    # the reported residual is the true FP64 one (Eq. 22)
    assert abs(osv.relres(F.apply, u0, host(x).reshape(u0.shape)) - rr) < 1e-9


@pytest.mark.parametrize("precision,tol,bar", [(lsm.LSM_FP64, 1e-11, 1e-9), (lsm.LSM_MIXED, 1e-8, 1e-6)])
def test_solve_batched_frequencies_and_sources(precision, tol, bar):
    """2 frequencies x 2 sources in one batched solve, each system against the oracle."""
    med = sy.random_medium((10, 12, 9), h=10.0, seed=7, frac=0.1)
    ws = [2 * np.pi * 6.0, 2 * np.pi * 14.0]
    h0 = handle(med, ws[0], precision=precision, tol=tol)
    h1 = lsm.lsm_create_shared(h0, ws[1])
    srcs = [(sy.explosion(), np.array([44.0, 51.0, 37.0])), (sy.double_couple_13(), np.array([31.0, 62.0, 45.0]))]
    hs, bs, xs, want = [], [], [], []
    for hh, w in ((h0, ws[0]), (h1, ws[1])):
        for M, s in srcs:
            b = torch.empty(3 * hh.N, dtype=torch.complex128, device="cuda")
            lsm.lsm_source(hh, M, s, b)
            hs.append(hh)
            bs.append(b)
            xs.append(torch.zeros_like(b))
            u0, _ = osrc.background_field(med.n, med.h, M, s, w, med.lam0, med.mu0, med.rho0)
            xo, *_ = osv.bicgstab(op.FFTOperator(med, w).apply, u0, tol=1e-13, maxit=400)
            want.append(xo)
    code, its, rrs, sts = lsm.lsm_solve_batched(hs, bs, xs)
    assert code == lsm.LSM_OK and all(s == 0 for s in sts)
    for x, xo, rr in zip(xs, want, rrs):
        assert rr <= tol
        assert rel(host(x).reshape(xo.shape), xo) < bar


@pytest.mark.parametrize("precision,tol", [(lsm.LSM_FP64, 1e-11), (lsm.LSM_MIXED, 1e-8)])
def test_graph_replay_matches_eager_launches(precision, tol):
    """The BiCGSTAB iterations replayed from a captured CUDA graph give bitwise the iterates of
    host-launched kernels (same kernels, same order, deterministic reductions); the graph is
    reused by a second solve, and the stage timer still sees every apply.  The library's launch
    count includes the replayed graphs' kernels: it stays close to the host-launched count (a
    replay runs two iterations, so it may launch one more iteration's kernels per inner solve,
    and it reads the host's control values back once per replay instead of once per iteration)."""
    med = sy.random_medium((12, 10, 9), h=10.0, seed=31, frac=0.1)
    srcs = [(sy.explosion(), np.array([44.0, 41.0, 37.0])), (sy.double_couple_12(), np.array([31.0, 52.0, 45.0])),
            (sy.double_couple_13(), np.array([61.0, 22.0, 45.0]))]
    out = {}
    for graph in (0, 1):
        h = handle(med, 2 * np.pi * 9.0, precision=precision, tol=tol, graph=graph)
        bs = []
        for M, s in srcs:
            b = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
            lsm.lsm_source(h, M, s, b)
            bs.append(b)
        runs = []
        for rep in range(2):
            lsm.lsm_timer_start(h, True)
            xs = [torch.zeros_like(b) for b in bs]
            n0 = lsm.lsm_launch_count(h)
            code, its, rrs, sts = lsm.lsm_solve_batched([h] * len(bs), bs, xs)
            nk = lsm.lsm_launch_count(h) - n0
            assert code == lsm.LSM_OK and all(r <= tol for r in rrs)
            ms, launches, applies = lsm.lsm_timer_read(h)
            runs.append((torch.stack(xs).cpu(), its, rrs, applies, nk))
            assert sum(launches) > 0 and sum(ms) > 0
        assert torch.equal(runs[0][0], runs[1][0]) and runs[0][1] == runs[1][1]
        out[graph] = runs[0]
    assert torch.equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2]
    assert tuple(out[0][3]) == tuple(out[1][3])   # executed system applies per precision
    assert out[0][4] > 0 and 0.8 * out[0][4] <= out[1][4] <= 1.25 * out[0][4] + 30


def test_solve_zero_rhs_and_noconv():
    med = sy.random_medium((8, 8, 8), h=10.0, seed=8, frac=0.1)
    h = handle(med, W, maxit=1, tol=1e-14)
    b = torch.zeros(3 * h.N, dtype=torch.complex128, device="cuda")
    x = dev(field(med.shape, 9)).reshape(-1)
    code, it, rr = lsm.lsm_solve(h, b, x, check=False)
    assert code == lsm.LSM_OK and it == 0
    assert torch.count_nonzero(x).item() == 0   # b = 0 gives x = 0 whatever the guess
    # one iteration cannot reach 1e-14: NOCONV with the last iterate returned
    lsm.lsm_source(h, sy.explosion(), [35.0, 35.0, 35.0], b)
    x.zero_()
    code, it, rr = lsm.lsm_solve(h, b, x, check=False)
    assert code == lsm.LSM_ERR_NOCONV and it == 1
    u0 = host(b).reshape(3, 8, 8, 8)
    rr_o = osv.relres(op.FFTOperator(med, W).apply, u0, host(x).reshape(u0.shape))
    assert abs(rr_o - rr) < 1e-12 and rr < 1.0


@pytest.mark.parametrize("precision", [lsm.LSM_FP64, lsm.LSM_MIXED])
def test_taper_parity(precision):
    """Eq. 25 absorbing taper applied by the library equals the oracle operator of the tapered medium,
    also after lsm_set_contrast."""
    med = sy.random_medium((16, 12, 10), h=8.0, seed=63, frac=0.2)
    h = handle(med, W, precision=precision, taper=4)
    t = op.tapered(med, 4)
    u = field(med.shape, 64)
    Au = torch.empty(3 * h.N, dtype=torch.complex128, device="cuda")
    lsm.lsm_apply(h, dev(u).reshape(-1), Au)
    want = op.FFTOperator(t, W).apply(u)
    assert rel(host(Au).reshape(u.shape), want) < 1e-12
    med2 = sy.random_medium((16, 12, 10), h=8.0, seed=65, frac=0.2)
    lsm.lsm_set_contrast(h, dev(med2.dC), dev(med2.drho))
    lsm.lsm_apply(h, dev(u).reshape(-1), Au)
    want2 = op.FFTOperator(op.tapered(med2, 4), W).apply(u)
    assert rel(host(Au).reshape(u.shape), want2) < 1e-12


def test_time_traces_parity():
    """Receiver traces (Ricker, inverse Fourier sum over +-f) against the oracle's synthesis."""
    from oracle import synthesis as osyn
    rng = np.random.default_rng(66)
    nf, ntr, nt, dt, df = 300, 7, 400, 3e-4, 1.25
    U = rng.standard_normal((nf, ntr)) + 1j * rng.standard_normal((nf, ntr))
    got = lsm.lsm_time_traces(dev(U), df, nt, dt, 60.0, 0.03)
    want = osyn.traces(U, df, nt, dt, 60.0, 0.03)
    assert np.abs(host(got) - want.reshape(ntr, nt)).max() < 1e-12 * np.abs(want).max()
