#!/usr/bin/env python
"""Benchmark of the matrix-free elastic Lippmann-Schwinger solve on GB300.

Workload (default "grf128_batched"): 128^3 grid, dx = 8 m, isotropic background
(vp 3000, vs 1730 m/s, rho 2300 kg/m^3) plus a seeded Gaussian-random-field
orthorhombic contrast (5% std, 40 m correlation; all 21 stiffness entries
stored and processed), 32 frequencies 2-40 Hz x 8 random unit-norm moment
tensors at the centre: 256 independent systems, solved to relative residual
1e-6 with the mixed-precision BiCGSTAB (FP32 operator applies, FP64-accurate
inner products and scalars, outer residual b - A x from an FP64 operator apply,
iterative refinement in FP64 storage).

The 256 systems run in memory waves: one wave = 8 consecutive frequencies x 8
tensors = 64 systems in one batched solve (every kernel launch covers all 64).
One step = one wave: its 64 moment-tensor background fields (Eqs. 13-16) and
its batched solve.  Warm-up steps and timed steps both start at the first wave
and cycle through the four, so K timed steps cover all 32 frequencies K/4 times
each when K is a multiple of 4.  The Green spectrum of each frequency is built
before timing (set up once per frequency, shared by its sources).

value = LS operator applications (system-level matvecs: FP32 inner applies plus
FP64 residual applies) per second over the whole job; solves/s beside it.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LS matvecs/s and solves/s at 128³ (FP32+refine vs FP64), % of HBM roofline"
STAGES = {0: "k_stress", 1: "k_divq+x fft", 2: "y fft", 3: "z fft+green", 4: "y ifft", 5: "x ifft+epilogue"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4, help="timed waves (a multiple of 4 covers every frequency equally)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grf128_batched")
    ap.add_argument("--grid", type=int, default=None, help="override the grid size (small profiling cases)")
    ap.add_argument("--freqs", type=int, default=None, help="use only the first F frequencies (profiling cases)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--systems", type=int, default=8, help="moment tensors per frequency")
    ap.add_argument("--wave-freqs", type=int, default=8, help="frequencies per memory wave (one batched solve)")
    ap.add_argument("--inner-tol", type=float, default=None, help="floor of the FP32 inner tolerance (mixed)")
    ap.add_argument("--maxit", type=int, default=2000, help="BiCGSTAB iteration limit (per inner solve when mixed)")
    ap.add_argument("--max-outer", type=int, default=None, help="mixed: refinement steps limit")
    ap.add_argument("--kernel", default="diff", choices=["diff", "h"],
                    help="operator form: difference form (default) or sampled analytic H (Eq. 21 literally)")
    ap.add_argument("--residual", default="fp64", choices=["fp64", "df"],
                    help="mixed: arithmetic of the outer residual's apply (FP64, or double-float pairs)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default FFT schedule (no autotuning)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-df-residual", action="store_true",
                    help="skip the side measurement of the mixed solve with the double-float residual apply")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparator (context only)")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------------------------
# algorithmic bytes of each apply stage, per system apply (b: bytes per complex, c: per real;
# share: systems of one launch that use the same Green spectrum, which the z pass stages once
# per block for all of them)
# --------------------------------------------------------------------------------------------
def stage_bytes(stage, n, b, c, share=1):
    nx, ny, nz = n
    N = nx * ny * nz
    Lx, Ly = 2 * nx, 2 * ny
    ex, ey, ez = nx + 2, ny + 2, nz + 2
    NO = (nx + 1) * (ny + 1) * (nz + 1)
    E = ex * ey * ez
    return {
        0: (3 * b + 21 * c + 6 * b) * N,
        1: 9 * N * b + N * c + 6 * E * b + 3 * ez * ey * Lx * b,
        2: 3 * ez * ey * Lx * b + 3 * ez * Ly * Lx * b,
        3: 3 * ez * Ly * Lx * b + 6 * NO * b / share + 3 * nz * Ly * Lx * b,
        4: 3 * nz * Ly * Lx * b + 3 * nz * ny * Lx * b,
        5: 3 * nz * ny * Lx * b + 3 * N * b + 3 * N * b,
    }[stage]


def stage_bytes_h(stage, n, b, c, share=1):
    """Algorithmic bytes of the sampled-H form's stages (9 transformed planes, 24 spectra)."""
    nx, ny, nz = n
    N = nx * ny * nz
    Lx, Ly, Lz = 2 * nx, 2 * ny, 2 * nz
    P = Lx * Ly * Lz
    NO = (nx + 1) * (ny + 1) * (nz + 1)
    return {
        0: (15 * b + 22 * c) * N,
        1: 9 * N * b + 9 * nz * ny * Lx * b,
        2: 9 * nz * ny * Lx * b + 9 * nz * Ly * Lx * b,
        3: 9 * nz * Ly * Lx * b + 9 * P * b + (9 * P + 24 * NO + 3 * P) * b + 3 * P * b + 3 * nz * Ly * Lx * b,
        4: 3 * nz * Ly * Lx * b + 3 * nz * ny * Lx * b,
        5: 3 * nz * ny * Lx * b + 3 * N * b + 3 * N * b,
    }[stage]


def stage_flops_h(stage, n):
    nx, ny, nz = n
    N = nx * ny * nz
    Lx, Ly, Lz = 2 * nx, 2 * ny, 2 * nz
    fft = lambda L: 5.0 * L * math.log2(L)  # noqa: E731
    return {
        0: N * (9 * 2 + 36 * 4) + 3 * N * 2,
        1: 9 * ny * nz * fft(Lx),
        2: 9 * nz * Lx * fft(Ly),
        3: (9 + 3) * Lx * Ly * fft(Lz) + Lx * Ly * Lz * (27 * 6 + 24 * 2),
        4: 3 * nz * Lx * fft(Ly),
        5: 3 * ny * nz * fft(Lx) + 3 * N * 2,
    }[stage]


def stage_flops(stage, n):
    """Model flops per system apply: 5 L log2 L per complex FFT line, 6 per complex multiply,
    2 per complex add, 4 per real-by-complex multiply-add."""
    nx, ny, nz = n
    N = nx * ny * nz
    Lx, Ly, Lz = 2 * nx, 2 * ny, 2 * nz
    ex, ey, ez = nx + 2, ny + 2, nz + 2
    fft = lambda L: 5.0 * L * math.log2(L)  # noqa: E731
    return {
        0: N * (9 * 2 + 36 * 4),
        1: ex * ey * ez * 3 * (6 * 2 + 2 + 4) + 3 * ey * ez * fft(Lx),
        2: 3 * ez * Lx * fft(Ly),
        3: 2 * 3 * Lx * Ly * fft(Lz) + Lx * Ly * Lz * (9 * 6 + 6 * 2),
        4: 3 * nz * Lx * fft(Ly),
        5: 3 * ny * nz * fft(Lx) + 3 * N * 2,
    }[stage]


# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA per clock per SM (1/64 of the
# 128 FP32 lanes) x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 pipe: 152 SMs x 128 FMA per clock x 2 flops x 2.07 GHz (the double-float stages run there)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_records():
    """Records of profiles/roofline_traffic.txt: 'key: value' lines, a new record at each 'stage:'."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    recs = []
    if not os.path.exists(path):
        return recs
    with open(path) as f:
        for line in f:
            if ":" not in line or line.startswith("#"):
                continue
            k, v = (x.strip() for x in line.split(":", 1))
            if k == "stage":
                recs.append({})
            if recs:
                recs[-1][k] = v
    return recs


def traffic_from_profile(stage, precision, n, share=None):
    """DRAM bytes per system apply of a stage from the committed ncu summary, if one matches the
    stage, the precision, the current kernel sources and (when the record names one) the number of
    systems sharing a spectrum; scaled to grid n by its voxels."""
    want_src = _csrc_digest()
    for rec in traffic_records():
        try:
            if int(rec["stage"]) != stage or rec["precision"] != precision or rec["csrc_sha256"] != want_src:
                continue
            if share is not None and "share" in rec and int(rec["share"]) != share:
                continue
            scale = (n[0] * n[1] * n[2]) / float(rec["grid_voxels"])
            return float(rec["dram_bytes_per_system_apply"]) * scale
        except (KeyError, ValueError):
            continue
    return None


def _csrc_digest():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2301_12836_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


# --------------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="lsm_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, operator applies of the same workload
# --------------------------------------------------------------------------------------------
def oracle_apply_sample(med, omega, reps=1, workers=None):
    """Time `reps` oracle applies (one thread: numpy.fft; workers = k: scipy.fft on k threads)."""
    from oracle import operator as op
    t0 = time.perf_counter()
    F = op.FFTOperator(med, omega, workers=workers)
    setup = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3,) + med.shape) + 1j * rng.standard_normal((3,) + med.shape)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        F.apply(u)
        times.append(time.perf_counter() - t0)
    return setup, times, F, u


def freq_blocks(nfreq, per_wave):
    """Consecutive frequency indices per memory wave."""
    return [list(range(i, min(i + per_wave, nfreq))) for i in range(0, nfreq, per_wave)]


def rank_blocks(rank, world, steps, nblocks):
    """Wave (block) index of each step on one rank: every rank cycles through all the waves, rank r
    starting at wave r, so all ranks do the same mix of work (weak scaling, replicas) and, while
    world <= nblocks, work on different frequencies at any one step.  No data is exchanged."""
    return [(rank + s) % nblocks for s in range(steps)]


def rank_frequencies(rank, world, steps, nfreq, per_wave=1):
    """Frequency indices a rank solves over `steps` waves (flattened)."""
    blocks = freq_blocks(nfreq, per_wave)
    return [f for b in rank_blocks(rank, world, steps, len(blocks)) for f in blocks[b]]


def reduce_timing(ms, applies, solves, launches, world, dist=None, device="cpu"):
    """Whole-job totals: the slowest rank's time, the sums of the work counters."""
    import torch
    t = torch.tensor([ms, applies, solves, launches], dtype=torch.float64, device=device)
    if world > 1:
        mx = t[:1].clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t[1:].clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        return float(mx[0]), float(sm[0]), float(sm[1]), float(sm[2])
    return float(t[0]), float(t[1]), float(t[2]), float(t[3])


def workload_inputs(args):
    import synthetic as sy
    wl = sy.get_workload(args.workload)
    n = args.grid or wl.n
    if args.grid:
        med = sy.grf_orthorhombic_medium(n, wl.h) if args.workload.startswith("grf") else sy.random_medium(n, wl.h)
    else:
        med = wl.medium()
    M, xs = wl.sources()
    c = (n - 1) / 2.0 * wl.h
    if args.grid:
        xs = np.repeat(np.array([[c, c, c]]), len(M), axis=0)
    k = min(args.systems, len(M))
    if k < args.systems:
        rng = np.random.default_rng(sy.BASE_SEED + 77)
        M = np.concatenate([M, sy.random_moment_tensors(args.systems - k, rng)])
        xs = np.repeat(xs[:1], args.systems, axis=0)
    freqs = list(wl.freqs_hz)[:args.freqs] if args.freqs else list(wl.freqs_hz)
    return wl, med, M[:args.systems], xs[:args.systems], freqs


def run_reference(args, rank, world):
    """The oracle, timed on the host cores: each step one LS apply of the workload (one thread)."""
    if rank != 0:
        return
    wl, med, M, xs, freqs = workload_inputs(args)
    omega = 2 * np.pi * freqs[0]
    setup, times, _, _ = oracle_apply_sample(med, omega, reps=args.warmup + args.steps)
    timed = times[args.warmup:]
    T = sum(timed)
    value = len(timed) / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(timed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, wl, med, freqs),
        "cpu_baseline": {"value": value, "unit": "matvec/s", "cores": 1, "kind": "oracle",
                         "sample": f"one FP64 NumPy FFT apply of the {med.n[0]}^3 workload per step "
                                   f"(operator setup {setup:.1f} s untimed)"},
        "e2e": {"value": value, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, wl, med, freqs):
    nb = len(freq_blocks(len(freqs), args.wave_freqs))
    return {"workload": wl.name if not args.grid else f"{wl.name}@{args.grid}", "grid": list(med.n), "dx_m": med.h,
            "frequencies_hz": f"{freqs[0]:g}-{freqs[-1]:g} ({len(freqs)})", "tensors_per_frequency": args.systems,
            "systems": len(freqs) * args.systems,
            "wave": {"systems": min(args.wave_freqs, len(freqs)) * args.systems,
                     "frequencies": min(args.wave_freqs, len(freqs)), "waves": nb,
                     "step": "one wave: its source fields and one batched solve of all its systems"},
            "timed_passes_over_all_frequencies": round(args.steps / nb, 3),
            "precision": args.precision, "kernel": args.kernel, "tol": wl.tol, "parallelism": "replicas",
            "residual": args.residual if args.precision == "mixed" else None,
            "l2": "inputs larger than L2 (contrast, Green spectra and Krylov vectors exceed 126 MB)"}


class Runner:
    """Handles of one medium at every frequency, the wave buffers, and the step of the hot path."""

    def __init__(self, lsm, torch, med, M, xs, freqs, blocks, nsys, opts, schedule=None):
        self.lsm, self.torch = lsm, torch
        self.M, self.xs = M, xs
        self.freqs, self.blocks, self.nsys = freqs, blocks, nsys
        dC = torch.from_numpy(med.dC).cuda().contiguous()
        drho = torch.from_numpy(med.drho).cuda().contiguous()
        self.handles = {}
        self.base = lsm.lsm_create(med.n, med.h, med.lam0, med.mu0, med.rho0, dC, drho, 2 * np.pi * freqs[0], opts)
        self.handles[0] = self.base
        for i in range(1, len(freqs)):
            self.handles[i] = lsm.lsm_create_shared(self.base, 2 * np.pi * freqs[i])
        del dC, drho
        if schedule is not None:
            lsm.lsm_set_schedule(self.base, lsm.LSM_FP64, schedule["fp64"])
            if opts.precision == lsm.LSM_MIXED:
                lsm.lsm_set_schedule(self.base, lsm.LSM_MIXED, schedule["fp32"])
        self.N3 = 3 * self.base.N
        self.wave = max(len(b) for b in blocks) * nsys
        self.b = [torch.empty(self.N3, dtype=torch.complex128, device="cuda") for _ in range(self.wave)]
        self.x = [torch.zeros(self.N3, dtype=torch.complex128, device="cuda") for _ in range(self.wave)]
        self.same_xs = bool(np.all(xs == xs[:1]))
        self.iters, self.relres = [], []

    def launches(self):
        return sum(self.lsm.lsm_launch_count(h) for h in self.handles.values())

    def step(self, blk, xset=None):
        lsm = self.lsm
        xset = self.x if xset is None else xset
        hs = []
        for j, f in enumerate(self.blocks[blk]):
            h = self.handles[f]
            out = self.b[j * self.nsys:(j + 1) * self.nsys]
            # moment tensors that share a position go through one source launch
            if self.same_xs:
                lsm.lsm_source_moments(h, self.M, self.xs[0], out)
            else:
                for k in range(self.nsys):
                    lsm.lsm_source(h, self.M[k], self.xs[k], out[k])
            hs += [h] * self.nsys
        k = len(hs)
        for v in xset[:k]:
            v.zero_()
        code, its, rrs, sts = lsm.lsm_solve_batched(hs, self.b[:k], xset[:k], check=False)
        if code != lsm.LSM_OK:
            raise RuntimeError(f"solve failed: {lsm.STATUS_NAMES.get(code)} {sts} relres {rrs}")
        self.iters.extend(its)
        self.relres.extend(rrs)
        return k

    def timed(self, seq):
        """CUDA-event time (ms) of the steps seq on the current stream; returns (ms, solves)."""
        torch = self.torch
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        solves = 0
        for blk in seq:
            solves += self.step(blk)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), solves

    def close(self):
        self.handles.clear()
        self.base = None
        self.b = self.x = None
        gc.collect()


def fused_epilogue(n, precision, kernel, schedule):
    """True when the FP32 inverse-x epilogue also sums the BiCGSTAB iteration's inner products
    (lsm_opts.fused_dots, on by default): mixed solves on an x side of 8, 32 or 128 whose inverse-x
    pass keeps its default schedule.  Then the applies v = A p (half the FP32 applies) also read
    r^ (one more vector of 3 N complex64)."""
    if precision != "mixed" or 2 * n[0] not in (16, 64, 256):
        return False
    v = 0 if (kernel == "h" or schedule is None) else schedule["fp32"][5]
    return v not in (1, 2)


def stage_records(lsm, st_ms, st_launch, a64, a32, ms, n, kernel, pair, share, fused=False):
    """Per-stage rooflines: FP32 stages against HBM (algorithmic bytes), FP64 stages against the
    FP64 pipe (model flops); double-float stages (FP32 pipe) against the HBM floor of their bytes
    with their FP64-equivalent rate.  fused: see fused_epilogue."""
    peak, _ = peaks()
    stages = []
    for slot in range(12):
        if st_launch[slot] == 0 or st_ms[slot] <= 0:
            continue
        f32 = slot >= 6
        stage = slot % 6
        napp = a32 if f32 else a64
        if napp == 0:
            continue
        name = STAGES[stage] + ("<float>" if f32 else ("<dfloat>" if pair else "<double>"))
        rec = {"kernel": name, "ms": round(st_ms[slot], 3), "launches": st_launch[slot],
               "share_of_step": round(st_ms[slot] / ms, 4), "system_applies": napp}
        sb, sf = (stage_bytes_h, stage_flops_h) if kernel == "h" else (stage_bytes, stage_flops)
        if f32:
            nbytes = sb(stage, n, 8, 4, share)
            if stage == 5 and fused:
                nbytes += 3 * n[0] * n[1] * n[2] * 8 / 2   # r^, read by half the applies
            ach = nbytes * napp / (st_ms[slot] / 1e3) / 1e9
            rec.update({"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4), "algorithmic_bytes_per_system_apply": round(nbytes)})
        elif pair:
            fl = sf(stage, n)
            nbytes = sb(stage, n, 16, 8, share)
            gbs = nbytes * napp / (st_ms[slot] / 1e3) / 1e9
            rec.update({"bound": "alu (FP32 pipe, double-float)", "achieved": round(gbs, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(gbs / peak, 4), "algorithmic_bytes_per_system_apply": round(nbytes),
                        "fp64_equivalent_tflops": round(fl * napp / (st_ms[slot] / 1e3) / 1e12, 4),
                        "model_flops_per_system_apply": fl})
        else:
            fl = sf(stage, n)
            ach = fl * napp / (st_ms[slot] / 1e3) / 1e12
            nbytes = sb(stage, n, 16, 8, share)
            rec.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                        "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                        "model_flops_per_system_apply": fl,
                        "hbm_gbs": round(nbytes * napp / (st_ms[slot] / 1e3) / 1e9, 1),
                        "algorithmic_bytes_per_system_apply": round(nbytes)})
        if kernel == "diff":
            t = traffic_from_profile(stage, "mixed" if f32 else ("dfloat" if pair else "fp64"), n, share)
            if t is not None:
                rec["traffic"] = round(t)
                rec["traffic_over_algorithmic"] = round(t / rec["algorithmic_bytes_per_system_apply"], 3)
        stages.append(rec)
    stages.sort(key=lambda r: -r["ms"])
    return stages


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    from paper_2301_12836_gb300 import lsm

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lsm.load()
    wl, med, M, xs, freqs = workload_inputs(args)
    nsys = args.systems
    prec = lsm.LSM_MIXED if args.precision == "mixed" else lsm.LSM_FP64
    pair = prec == lsm.LSM_MIXED and args.residual == "df"
    blocks = freq_blocks(len(freqs), args.wave_freqs)
    nb = len(blocks)
    warm_seq = rank_blocks(rank, world, args.warmup, nb)
    timed_seq = rank_blocks(rank, world, args.steps, nb)
    kern = lsm.LSM_KERNEL_H if args.kernel == "h" else lsm.LSM_KERNEL_DIFF

    def mk_opts(precision, residual):
        o = lsm.lsm_default_opts(precision=precision, tol=wl.tol, maxit=args.maxit, kernel=kern,
                                 residual=lsm.LSM_RESIDUAL_DFLOAT if residual == "df" else lsm.LSM_RESIDUAL_FP64)
        if args.inner_tol:
            o.inner_tol = args.inner_tol
        if args.max_outer:
            o.max_outer = args.max_outer
        return o

    t_setup = time.perf_counter()
    R = Runner(lsm, torch, med, M, xs, freqs, blocks, nsys, mk_opts(prec, args.residual))
    schedule = None
    if not args.no_tune:
        v64, v32 = lsm.lsm_autotune(R.base, nsys, 2)
        schedule = {"fp64": v64, "fp32": v32}
    # pinned host buffers for the e2e measurement, allocated and written here at setup: pinning
    # 12.8 GB and first writes into it keep the host busy for a while, which slowed the e2e loop's
    # latency-bound host side when it came right before it
    host = None
    if not args.no_e2e:
        host = [[torch.empty(R.N3, dtype=torch.complex128, pin_memory=True) for _ in range(R.wave)] for _ in range(2)]
        for k in range(2):
            for j in range(R.wave):
                host[k][j].copy_(R.x[j])
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    for blk in warm_seq:
        R.step(blk)
    R.iters, R.relres = [], []
    launches0 = R.launches()
    lsm.lsm_timer_start(R.base, True)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with sampler:
        time.sleep(0.3)
        ms, solves = R.timed(timed_seq)
    if world > 1:
        dist.barrier()
    st_ms, st_launch, (a64, a32) = lsm.lsm_timer_read(R.base)
    launches = R.launches() - launches0
    applies = a64 + a32
    ms_max, applies_all, solves_all, launches_all = reduce_timing(ms, applies, solves, launches, world, dist, "cuda")
    value = applies_all / (ms_max / 1e3)
    stages = stage_records(lsm, st_ms, st_launch, a64, a32, ms, med.n, args.kernel, pair, nsys,
                           fused_epilogue(med.n, args.precision, args.kernel, schedule))
    dom = dict(stages[0]) if stages else {}
    if dom:
        prec_s = "mixed" if dom["kernel"].endswith("<float>") else ("dfloat" if dom["kernel"].endswith("<dfloat>") else "fp64")
        stage_id = [k for k, v in STAGES.items() if dom["kernel"].startswith(v)][0]
        dom["traffic"] = traffic_from_profile(stage_id, prec_s, med.n, nsys) if args.kernel == "diff" else None
        dom["peak_kind"] = ("measured" if peaks()[1] == "measured" else "fallback") if dom["unit"] == "GB/s" else \
            "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"
    timed_freqs = sorted({f for blk in timed_seq for f in blocks[blk]})
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "matvec/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("f32+df64" if pair else "f32+f64") if prec == lsm.LSM_MIXED else "f64",
        "data": "synthetic", "config": _config(args, wl, med, freqs),
        "timed_frequencies": len(timed_freqs),
        "solves_per_s": round(solves_all / (ms_max / 1e3), 4),
        "matvecs": {"fp32": a32, "residual": a64, "residual_arith": "df64" if pair else "f64",
                    "per_solve": round(applies / solves, 2), "residual_per_solve": round(a64 / solves, 3)},
        "iterations_mean": round(float(np.mean(R.iters)), 2),
        "relres_max": float(np.max(R.relres)),
        "setup_s": round(t_setup, 2),
        "schedule": schedule,
        "roofline": dom, "stages": stages, "gpu_launches": int(launches_all),
    }
    cs = sampler.summary()
    if cs:
        line["clocks"] = cs

    # end to end through the C ABI with host buffers: every wave's solutions are copied to pinned
    # host memory inside the timed region.  Two solution sets alternate, and each set's copy runs
    # on a copy stream while the next wave solves into the other set; a set is reused only after
    # its copy has finished.
    if not args.no_e2e:
        xsets = [R.x, [torch.zeros_like(v) for v in R.x]]
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        lsm.lsm_timer_start(R.base, False)
        # untimed copies into every pinned buffer from the copy stream: the first transfers into
        # freshly pinned pages measured slow while kernels ran beside them
        for _ in range(2):
            with torch.cuda.stream(copy_stream):
                for k in range(2):
                    for j in range(R.wave):
                        host[k][j].copy_(xsets[k][j], non_blocking=True)
            copy_stream.synchronize()
        # one untimed step: the solver's iteration graph is captured per stage-timer state
        R.step(timed_seq[0], xsets[1])
        lsm.lsm_timer_start(R.base, False)   # same timer state; zeroes the apply counters
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_solves = 0
        d2h = 0
        for i, blk in enumerate(timed_seq):
            k = i % 2
            cur = torch.cuda.current_stream()
            cur.wait_event(copied[k])
            ns = R.step(blk, xsets[k])
            e_solves += ns
            d2h += ns * R.N3 * 16
            solved = torch.cuda.Event()
            solved.record(cur)
            copy_stream.wait_event(solved)
            with torch.cuda.stream(copy_stream):
                for j in range(ns):
                    host[k][j].copy_(xsets[k][j], non_blocking=True)
            copied[k].record(copy_stream)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        _, _, (e64, e32) = lsm.lsm_timer_read(R.base)
        line["e2e"] = {"value": round((e64 + e32) / te, 3), "unit": "matvec/s",
                       "h2d_bytes_per_step": R.wave * 9 * 8, "d2h_bytes_per_step": round(d2h / len(timed_seq)),
                       "solves_per_s": round(e_solves / te, 4)}
        del host, xsets, copy_stream

    # context, outside the timed region: cuFFT (through torch.fft) doing only the forward and
    # inverse 3-D transforms of the three padded components of one FP32 apply (no pruning, no
    # contraction, no Green multiply), against this library's FFT stages 1-5 of the same apply
    # (which also form the divergence, skip the padding, multiply by the spectrum and crop)
    if rank == 0 and not args.no_cufft and args.kernel == "diff" and a32:
        L = [2 * v for v in med.n]
        buf = torch.zeros((3, L[2], L[1], L[0]), dtype=torch.complex64, device="cuda")
        for _ in range(2):
            torch.fft.ifftn(torch.fft.fftn(buf, dim=(-3, -2, -1)), dim=(-3, -2, -1))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 5
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            torch.fft.ifftn(torch.fft.fftn(buf, dim=(-3, -2, -1)), dim=(-3, -2, -1))
        e1.record()
        torch.cuda.synchronize()
        del buf
        ours = sum(st_ms[6 + k] for k in range(1, 6)) / a32
        line["cufft_comparator"] = {
            "cufft_fft_ifft_ms_per_system_apply": round(e0.elapsed_time(e1) / reps, 4),
            "ours_stages_1_5_ms_per_system_apply": round(ours, 4),
            "note": "complex64, 3 components, full (2n)^3 transforms vs pruned two-step passes with the "
                    "divergence, Green multiply and crop fused in; not part of the timed region"}
    R.close()
    torch.cuda.empty_cache()
    one_pass = list(range(nb))

    # side line: the same systems with the residual apply in double-float pairs (or in FP64 when
    # the headline used pairs), one pass over every wave after one untimed wave
    if prec == lsm.LSM_MIXED and not args.no_df_residual and rank == 0:
        other = "fp64" if pair else "df"
        S = Runner(lsm, torch, med, M, xs, freqs, blocks, nsys, mk_opts(prec, other), schedule)
        S.step(one_pass[0])
        S.iters, S.relres = [], []
        lsm.lsm_timer_start(S.base, False)
        tr, ns = S.timed(one_pass)
        _, _, (r64, r32) = lsm.lsm_timer_read(S.base)
        key = "fp64_residual" if other == "fp64" else "df_residual"
        line[key] = {"value": round((r64 + r32) / (tr / 1e3), 3), "unit": "matvec/s",
                     "solves_per_s": round(ns / (tr / 1e3), 4), "ms_per_step": round(tr / len(one_pass), 3),
                     "dtype": "f32+f64" if other == "fp64" else "f32+df64", "steps": len(one_pass),
                     "relres_max": float(np.max(S.relres)), "iterations_mean": round(float(np.mean(S.iters)), 2),
                     "residual_matvecs_per_solve": round(r64 / ns, 3),
                     "note": "the mixed solve with its outer residual apply in "
                             + ("FP64" if other == "fp64" else "double-float pairs (about 48 significand bits)")
                             + "; the same 256 systems, one pass, CUDA-event timed"}
        S.close()
        torch.cuda.empty_cache()

    # the plain FP64 GPU form on the same systems (all waves, one pass), for the precision
    # comparison at the same relative residual
    if prec == lsm.LSM_MIXED and not args.no_fp64_form and rank == 0:
        P = Runner(lsm, torch, med, M, xs, freqs, blocks, nsys, mk_opts(lsm.LSM_FP64, "fp64"), schedule)
        P.step(one_pass[0])
        P.iters, P.relres = [], []
        lsm.lsm_timer_start(P.base, False)
        tf, ns = P.timed(one_pass)
        _, _, (f64, _) = lsm.lsm_timer_read(P.base)
        line["fp64_form"] = {"solves_per_s": round(ns / (tf / 1e3), 4), "matvecs_per_s": round(f64 / (tf / 1e3), 3),
                             "ms_per_step": round(tf / len(one_pass), 3), "steps": len(one_pass), "solves": ns,
                             "iterations_mean": round(float(np.mean(P.iters)), 2),
                             "relres_max": float(np.max(P.relres)),
                             "note": "plain FP64 BiCGSTAB on the same systems (every frequency and tensor), "
                                     "one pass, CUDA-event timed"}
        P.close()
        torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        setup, times, F, u = oracle_apply_sample(med, 2 * np.pi * freqs[0], reps=1)
        ncores = os.cpu_count() or 1
        F.workers = ncores
        t0 = time.perf_counter()
        F.apply(u)
        t_all = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(1.0 / times[0], 5), "unit": "matvec/s", "cores": 1, "kind": "oracle",
                                "sample": f"one FP64 NumPy FFT apply of the {med.n[0]}^3 workload "
                                          f"({times[0]:.1f} s; operator setup {setup:.1f} s untimed)",
                                "all_cores": {"value": round(1.0 / t_all, 5), "unit": "matvec/s", "cores": ncores,
                                              "sample": f"the same apply with scipy.fft on {ncores} threads "
                                                        f"({t_all:.1f} s; the rest of the oracle is single-threaded)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
