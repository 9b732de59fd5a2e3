#!/usr/bin/env python
"""Benchmark of the matrix-free elastic Lippmann-Schwinger solve on GB300.

Workload (default "grf128_batched"): 128^3 grid, dx = 8 m, isotropic background
(vp 3000, vs 1730 m/s, rho 2300 kg/m^3) plus a seeded Gaussian-random-field
orthorhombic contrast (5% std, 40 m correlation; all 21 stiffness entries
stored and processed), 32 frequencies 2-40 Hz x 8 random unit-norm moment
tensors at the centre.  One step = the hot path for one frequency: the 8
moment-tensor background fields (Eqs. 13-16) and one batched mixed-precision
BiCGSTAB solve of the 8 systems (FP32 applies, FP64-accurate inner products,
outer residual in double-float arithmetic (pairs of FP32 words, about 48
significand bits) with FP64 storage, iterative refinement) to relative
residual 1e-6.  Consecutive steps take
consecutive frequencies.  The Green spectrum of each frequency is built before
timing (it is set up once per frequency and shared by all its sources).

value = LS operator applications (system-level matvecs, FP32 inner + outer residual) per second
over the whole job; solves/s is reported beside it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LS matvecs/s and solves/s at 128³ (FP32+refine vs FP64), % of HBM roofline"
STAGES = {0: "k_stress", 1: "k_divq+x fft", 2: "y fft", 3: "z fft+green", 4: "y ifft", 5: "x ifft+epilogue"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grf128_batched")
    ap.add_argument("--grid", type=int, default=None, help="override the grid size (small profiling cases)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--systems", type=int, default=8, help="moment tensors solved together per step")
    ap.add_argument("--inner-tol", type=float, default=None, help="floor of the FP32 inner tolerance (mixed)")
    ap.add_argument("--kernel", default="diff", choices=["diff", "h"],
                    help="operator form: difference form (default) or sampled analytic H (Eq. 21 literally)")
    ap.add_argument("--residual", default="df", choices=["df", "fp64"],
                    help="mixed: arithmetic of the outer residual's apply (double-float pairs or FP64)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default FFT schedule (no autotuning)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-fp64-residual", action="store_true",
                    help="skip the side measurement of the mixed solve with the FP64 residual apply")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparator (context only)")
    return ap.parse_args()


# --------------------------------------------------------------------------------------------
# algorithmic bytes of each apply stage, per system apply (b: bytes per complex, c: per real)
# --------------------------------------------------------------------------------------------
def stage_bytes(stage, n, b, c):
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
        3: 3 * ez * Ly * Lx * b + 6 * NO * b + 3 * nz * Ly * Lx * b,
        4: 3 * nz * Ly * Lx * b + 3 * nz * ny * Lx * b,
        5: 3 * nz * ny * Lx * b + 3 * N * b + 3 * N * b,
    }[stage]


def stage_bytes_h(stage, n, b, c):
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
    import math
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
    import math
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


def traffic_from_profile(stage, precision, n):
    """DRAM bytes per system apply of the timed stage from the committed ncu summary, if it matches."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if not os.path.exists(path):
        return None
    want_src = _csrc_digest()
    rec = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
    try:
        if (int(rec["stage"]) != stage or rec["precision"] != precision or rec["csrc_sha256"] != want_src):
            return None
        scale = (n[0] * n[1] * n[2]) / float(rec["grid_voxels"])
        return float(rec["dram_bytes_per_system_apply"]) * scale
    except (KeyError, ValueError):
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, one operator apply of the same workload
# --------------------------------------------------------------------------------------------
def oracle_apply_sample(med, omega, reps=1):
    from oracle import operator as op
    t0 = time.perf_counter()
    F = op.FFTOperator(med, omega)
    setup = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3,) + med.shape) + 1j * rng.standard_normal((3,) + med.shape)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        F.apply(u)
        times.append(time.perf_counter() - t0)
    return setup, times


def rank_frequencies(rank, world, steps_total, nfreq):
    """Frequencies (indices) a rank solves, one per step: ranks take disjoint consecutive blocks
    (weak scaling: every rank does the same work; no data is exchanged between ranks)."""
    return [(rank * steps_total + s) % nfreq for s in range(steps_total)]


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
    return wl, med, M[:args.systems], xs[:args.systems]


def run_reference(args, rank, world):
    """The oracle, timed on the host cores: each step one LS apply of the workload."""
    if rank != 0:
        return
    wl, med, M, xs = workload_inputs(args)
    omega = 2 * np.pi * wl.freqs_hz[0]
    setup, times = oracle_apply_sample(med, omega, reps=args.warmup + args.steps)
    timed = times[args.warmup:]
    T = sum(timed)
    value = len(timed) / T
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(timed), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, wl, med),
        "cpu_baseline": {"value": value, "unit": "matvec/s", "cores": 1, "kind": "oracle",
                         "sample": f"one FP64 NumPy FFT apply of the {med.n[0]}^3 workload per step "
                                   f"(operator setup {setup:.1f} s untimed)"},
        "e2e": {"value": value, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(args, wl, med):
    f = wl.freqs_hz
    return {"workload": wl.name if not args.grid else f"{wl.name}@{args.grid}", "grid": list(med.n), "dx_m": med.h,
            "frequencies_hz": f"{f[0]:g}-{f[-1]:g} ({len(f)})", "systems_per_step": args.systems,
            "precision": args.precision, "kernel": args.kernel, "tol": wl.tol, "parallelism": "replicas",
            "residual": args.residual if args.precision == "mixed" else None,
            "l2": "inputs larger than L2 (contrast, Green spectra and Krylov vectors exceed 126 MB)"}


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
    wl, med, M, xs = workload_inputs(args)
    nsys = args.systems
    prec = lsm.LSM_MIXED if args.precision == "mixed" else lsm.LSM_FP64
    steps_total = args.warmup + args.steps
    freqs = list(wl.freqs_hz)
    # weak scaling: rank r takes its own frequencies
    fidx = rank_frequencies(rank, world, steps_total, len(freqs))
    dC = torch.from_numpy(med.dC).cuda().contiguous()
    drho = torch.from_numpy(med.drho).cuda().contiguous()
    opts = lsm.lsm_default_opts(precision=prec, tol=wl.tol, maxit=2000,
                                kernel=lsm.LSM_KERNEL_H if args.kernel == "h" else lsm.LSM_KERNEL_DIFF,
                                residual=lsm.LSM_RESIDUAL_FP64 if args.residual == "fp64" else lsm.LSM_RESIDUAL_DFLOAT)
    if args.inner_tol:
        opts.inner_tol = args.inner_tol
    handles = {}
    t_setup = time.perf_counter()
    base = lsm.lsm_create(med.n, med.h, med.lam0, med.mu0, med.rho0, dC, drho, 2 * np.pi * freqs[fidx[0]], opts)
    handles[fidx[0]] = base
    for i in fidx:
        if i not in handles:
            handles[i] = lsm.lsm_create_shared(base, 2 * np.pi * freqs[i])
    del dC, drho
    schedule = None
    if not args.no_tune:
        v64, v32 = lsm.lsm_autotune(base, nsys, 2)
        schedule = {"fp64": v64, "fp32": v32}
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    N3 = 3 * base.N
    b = [torch.empty(N3, dtype=torch.complex128, device="cuda") for _ in range(nsys)]
    x = [torch.zeros(N3, dtype=torch.complex128, device="cuda") for _ in range(nsys)]
    stats = {"iters": [], "relres": []}
    same_xs = bool(np.all(xs == xs[:1]))

    def sources(h, out):
        # moment tensors that share a position go through one source launch
        if same_xs:
            lsm.lsm_source_moments(h, M, xs[0], out)
        else:
            for j in range(nsys):
                lsm.lsm_source(h, M[j], xs[j], out[j])

    def step(s, xs_=None):
        xs_ = x if xs_ is None else xs_
        h = handles[fidx[s]]
        sources(h, b)
        for j in range(nsys):
            xs_[j].zero_()
        code, its, rrs, sts = lsm.lsm_solve_batched([h] * nsys, b, xs_, check=False)
        if code != lsm.LSM_OK:
            raise RuntimeError(f"solve failed: {lsm.STATUS_NAMES.get(code)} {sts} relres {rrs}")
        stats["iters"].extend(its)
        stats["relres"].extend(rrs)

    for s in range(args.warmup):
        step(s)
    stats = {"iters": [], "relres": []}
    launches0 = sum(lsm.lsm_launch_count(h) for h in handles.values())
    lsm.lsm_timer_start(base, True)
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
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in range(args.warmup, steps_total):
            step(s)
        e1.record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    st_ms, st_launch, (a64, a32) = lsm.lsm_timer_read(base)
    launches = sum(lsm.lsm_launch_count(h) for h in handles.values()) - launches0
    solves = args.steps * nsys
    applies = a64 + a32
    ms_max, applies_all, solves_all, launches_all = reduce_timing(ms, applies, solves, launches, world, dist, "cuda")
    value = applies_all / (ms_max / 1e3)
    # per-stage rooflines: FP32 stages against HBM (algorithmic bytes), FP64 stages against the
    # FP64 pipe (model flops); the dominant stage (largest share of the timed region) is reported.
    # With the double-float residual (mixed) the FP64 slots time the pair apply:
    # its model flops are those of the FP64 form, each carried out as several FP32 operations, so
    # it is given against the HBM floor of its bytes and its FP64-equivalent rate, with no ALU frac.
    pair = prec == lsm.LSM_MIXED and args.residual == "df"
    peak, peak_kind = peaks()
    stages = []
    for slot in range(12):
        if st_launch[slot] == 0 or st_ms[slot] <= 0:
            continue
        f32 = slot >= 6
        stage = slot % 6
        napp = a32 if f32 else a64
        name = STAGES[stage] + ("<float>" if f32 else ("<dfloat>" if pair else "<double>"))
        rec = {"kernel": name, "ms": round(st_ms[slot], 3), "launches": st_launch[slot],
               "share_of_step": round(st_ms[slot] / ms, 4)}
        sb, sf = (stage_bytes_h, stage_flops_h) if args.kernel == "h" else (stage_bytes, stage_flops)
        if f32:
            nbytes = sb(stage, med.n, 8, 4)
            ach = nbytes * napp / (st_ms[slot] / 1e3) / 1e9
            rec.update({"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(ach / peak, 4), "algorithmic_bytes_per_system_apply": nbytes})
        elif pair:
            fl = sf(stage, med.n)
            nbytes = sb(stage, med.n, 16, 8)
            gbs = nbytes * napp / (st_ms[slot] / 1e3) / 1e9
            rec.update({"bound": "alu (FP32 pipe, double-float)", "achieved": round(gbs, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(gbs / peak, 4), "algorithmic_bytes_per_system_apply": nbytes,
                        "fp64_equivalent_tflops": round(fl * napp / (st_ms[slot] / 1e3) / 1e12, 4),
                        "model_flops_per_system_apply": fl})
        else:
            fl = sf(stage, med.n)
            ach = fl * napp / (st_ms[slot] / 1e3) / 1e12
            rec.update({"bound": "alu", "achieved": round(ach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                        "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                        "model_flops_per_system_apply": fl})
        stages.append(rec)
    stages.sort(key=lambda r: -r["ms"])
    dom = dict(stages[0]) if stages else {}
    if dom:
        prec_s = "mixed" if dom["kernel"].endswith("<float>") else ("dfloat" if dom["kernel"].endswith("<dfloat>") else "fp64")
        stage_id = [k for k, v in STAGES.items() if dom["kernel"].startswith(v)][0]
        dom["traffic"] = traffic_from_profile(stage_id, prec_s, med.n) if args.kernel == "diff" else None
        dom["peak_kind"] = peak_kind if dom["unit"] == "GB/s" else "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"
    roof = dom

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "matvec/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ("f32+df64" if pair else "f32+f64") if prec == lsm.LSM_MIXED else "f64",
        "data": "synthetic", "config": _config(args, wl, med),
        "solves_per_s": round(solves_all / (ms_max / 1e3), 4),
        "matvecs": {"fp32": a32, "residual": a64, "residual_arith": "df64" if pair else "f64",
                    "per_solve": round(applies / solves, 2)},
        "iterations_mean": round(float(np.mean(stats["iters"])), 2),
        "relres_max": float(np.max(stats["relres"])),
        "setup_s": round(t_setup, 2),
        "schedule": schedule,
        "roofline": roof, "stages": stages, "gpu_launches": int(launches_all),
    }
    cs = sampler.summary()
    if cs:
        line["clocks"] = cs

    # end to end through the C ABI with host buffers: every step's solutions are copied to pinned
    # host memory inside the timed region.  Two solution sets alternate, and each set's copy runs
    # on a copy stream while the next step solves into the other set; a set is reused only after
    # its copy has finished.
    if not args.no_e2e:
        host = [[torch.empty(N3, dtype=torch.complex128, pin_memory=True) for _ in range(nsys)] for _ in range(2)]
        xsets = [x, [torch.zeros_like(v) for v in x]]
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        lsm.lsm_timer_start(base, False)
        # one untimed copy into every pinned buffer: the first transfers into freshly pinned pages
        # measured slow while kernels ran beside them (on a box that had run other GPU jobs)
        with torch.cuda.stream(copy_stream):
            for k in range(2):
                for j in range(nsys):
                    host[k][j].copy_(xsets[k][j], non_blocking=True)
        copy_stream.synchronize()
        # one untimed step: the solver's iteration graph is captured per timer state, so the first
        # solve after switching the stage timer off re-captures it
        step(args.warmup, xsets[1])
        lsm.lsm_timer_start(base, False)   # same timer state; zeroes the apply counters
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i, s in enumerate(range(args.warmup, steps_total)):
            k = i % 2
            cur = torch.cuda.current_stream()
            cur.wait_event(copied[k])
            step(s, xsets[k])
            solved = torch.cuda.Event()
            solved.record(cur)
            copy_stream.wait_event(solved)
            with torch.cuda.stream(copy_stream):
                for j in range(nsys):
                    host[k][j].copy_(xsets[k][j], non_blocking=True)
            copied[k].record(copy_stream)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        _, _, (e64, e32) = lsm.lsm_timer_read(base)
        line["e2e"] = {"value": round((e64 + e32) / te, 3), "unit": "matvec/s",
                       "h2d_bytes_per_step": nsys * 9 * 8, "d2h_bytes_per_step": nsys * N3 * 16,
                       "solves_per_s": round(solves / te, 4)}

    # the same K steps with the mixed solve's residual apply in FP64 (LSM_RESIDUAL_FP64), timed the
    # same way (CUDA events, one untimed step first), beside the double-float headline
    if pair and not args.no_fp64_residual and rank == 0:
        dC = torch.from_numpy(med.dC).cuda().contiguous()
        drho = torch.from_numpy(med.drho).cuda().contiguous()
        o_r = lsm.lsm_default_opts(precision=prec, tol=wl.tol, maxit=2000, kernel=opts.kernel,
                                   residual=lsm.LSM_RESIDUAL_FP64)
        hr = {fidx[args.warmup]: lsm.lsm_create(med.n, med.h, med.lam0, med.mu0, med.rho0, dC, drho,
                                                2 * np.pi * freqs[fidx[args.warmup]], o_r)}
        del dC, drho
        rbase = hr[fidx[args.warmup]]
        for s in range(args.warmup, steps_total):
            if fidx[s] not in hr:
                hr[fidx[s]] = lsm.lsm_create_shared(rbase, 2 * np.pi * freqs[fidx[s]])
        if schedule is not None:
            lsm.lsm_set_schedule(rbase, lsm.LSM_FP64, schedule["fp64"])
            lsm.lsm_set_schedule(rbase, lsm.LSM_MIXED, schedule["fp32"])
        rr_max = []

        def rstep(s):
            h = hr[fidx[s]]
            sources(h, b)
            for j in range(nsys):
                x[j].zero_()
            code, its, rrs, sts = lsm.lsm_solve_batched([h] * nsys, b, x, check=False)
            if code != lsm.LSM_OK:
                raise RuntimeError(f"FP64-residual solve failed: {lsm.STATUS_NAMES.get(code)} {sts}")
            rr_max.append(max(rrs))

        rstep(args.warmup)
        lsm.lsm_timer_start(rbase, False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for s in range(args.warmup, steps_total):
            rstep(s)
        e1.record()
        torch.cuda.synchronize()
        tr = e0.elapsed_time(e1) / 1e3
        _, _, (r64, r32) = lsm.lsm_timer_read(rbase)
        line["fp64_residual"] = {"value": round((r64 + r32) / tr, 3), "unit": "matvec/s",
                                 "solves_per_s": round(solves / tr, 4), "ms_per_step": round(tr * 1e3 / args.steps, 3),
                                 "dtype": "f32+f64", "relres_max": float(np.max(rr_max[1:])),
                                 "note": "the mixed solve with its outer residual apply in FP64; same steps, "
                                         "timed with CUDA events"}
        del hr, rbase

    # the plain FP64 GPU form on the first frequency, for the precision comparison
    if prec == lsm.LSM_MIXED and not args.no_fp64_form and rank == 0:
        dC = torch.from_numpy(med.dC).cuda().contiguous()
        drho = torch.from_numpy(med.drho).cuda().contiguous()
        o64 = lsm.lsm_default_opts(precision=lsm.LSM_FP64, tol=wl.tol, maxit=2000, kernel=opts.kernel)
        h64 = lsm.lsm_create(med.n, med.h, med.lam0, med.mu0, med.rho0, dC, drho, 2 * np.pi * freqs[fidx[-1]], o64)
        del dC, drho
        if schedule is not None:
            lsm.lsm_set_schedule(h64, lsm.LSM_FP64, schedule["fp64"])
        sources(h64, b)
        for j in range(nsys):
            x[j].zero_()
        lsm.lsm_timer_start(h64, False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, its, rrs, sts = lsm.lsm_solve_batched([h64] * nsys, b, x, check=False)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        _, _, (f64, _) = lsm.lsm_timer_read(h64)
        line["fp64_form"] = {"solves_per_s": round(nsys / tf, 4), "matvecs_per_s": round(f64 / tf, 3),
                             "iterations_mean": float(np.mean(its)), "relres_max": float(np.max(rrs)),
                             "status": lsm.STATUS_NAMES.get(code), "frequency_hz": freqs[fidx[-1]]}
        del h64

    # context, outside the timed region: cuFFT (through torch.fft) doing only the forward and
    # inverse 3-D transforms of the three padded components of one FP32 apply (no pruning, no
    # contraction, no Green multiply), against this library's FFT stages 1-5 of the same apply
    # (which also form the divergence, skip the padding, multiply by the spectrum and crop)
    if rank == 0 and not args.no_cufft and args.kernel == "diff":
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
        ours = sum(st_ms[6 + k] for k in range(1, 6)) / a32 if a32 else None
        line["cufft_comparator"] = {
            "cufft_fft_ifft_ms_per_system_apply": round(e0.elapsed_time(e1) / reps, 4),
            "ours_stages_1_5_ms_per_system_apply": round(ours, 4) if ours else None,
            "note": "complex64, 3 components, full (2n)^3 transforms vs pruned two-step passes with the "
                    "divergence, Green multiply and crop fused in; not part of the timed region"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        setup, times = oracle_apply_sample(med, 2 * np.pi * freqs[fidx[0]], reps=1)
        line["cpu_baseline"] = {"value": round(1.0 / times[0], 5), "unit": "matvec/s", "cores": 1, "kind": "oracle",
                                "sample": f"one FP64 NumPy FFT apply of the {med.n[0]}^3 workload "
                                          f"({times[0]:.1f} s; operator setup {setup:.1f} s untimed)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
