"""Host-side helpers of bench.py (no GPU): the algorithmic byte model of one operator apply that
the roofline divides by, and the lookup of the pinned ncu DRAM traffic of the dominant kernel."""
import os

import bench

N128 = (128, 128, 128)


def test_stage_bytes_model_128():
    # per stage for the complex64 path (8-byte complex, 4-byte real), in MB: the kernel table's figures
    mb = [round(bench.stage_bytes(s, N128, 8, 4) / 1e6) for s in range(6)]
    assert mb == [327, 369, 308, 509, 302, 201]
    # complex128 / double-float pairs move exactly twice the bytes
    assert all(bench.stage_bytes(s, N128, 16, 8) == 2 * bench.stage_bytes(s, N128, 8, 4) for s in range(6))
    # the z pass stages each frequency's octant spectrum (6 x 129^3 complex) once for the systems of
    # a launch that share it: with 8 sources per frequency its bytes per system apply fall to 419 MB
    g = 6 * 129 ** 3 * 8
    assert bench.stage_bytes(3, N128, 8, 4, share=8) == bench.stage_bytes(3, N128, 8, 4) - g * 7 / 8
    assert round(bench.stage_bytes(3, N128, 8, 4, share=8) / 1e6) == 419
    assert all(bench.stage_bytes(s, N128, 8, 4, share=8) == bench.stage_bytes(s, N128, 8, 4) for s in (0, 1, 2, 4, 5))


def test_fused_epilogue_cases():
    """The FP32 inverse-x epilogue sums the iteration's inner products (and its v = A p applies
    read r^) for mixed solves on x sides 8, 32 and 128 with that pass's default schedule."""
    sched = {"fp64": [0] * 6, "fp32": [0] * 6}
    assert bench.fused_epilogue(N128, "mixed", "diff", sched)
    assert bench.fused_epilogue((32, 20, 24), "mixed", "diff", None)
    assert bench.fused_epilogue((8, 6, 10), "mixed", "h", {"fp64": [0] * 6, "fp32": [0, 0, 0, 0, 0, 1]})
    assert not bench.fused_epilogue(N128, "fp64", "diff", sched)
    assert not bench.fused_epilogue((96, 96, 96), "mixed", "diff", sched)
    assert not bench.fused_epilogue((64, 64, 64), "mixed", "diff", sched)
    assert not bench.fused_epilogue(N128, "mixed", "diff", {"fp64": [0] * 6, "fp32": [0, 0, 0, 0, 0, 2]})


def test_waves_cover_every_frequency():
    blocks = bench.freq_blocks(32, 8)
    assert blocks == [list(range(8 * k, 8 * k + 8)) for k in range(4)]
    assert bench.freq_blocks(10, 4) == [[0, 1, 2, 3], [4, 5, 6, 7], [8, 9]]
    # timed steps start at the first wave and cycle: 4 steps cover each of the 32 frequencies once
    seq = bench.rank_blocks(0, 1, 4, 4)
    assert sorted(f for b in seq for f in blocks[b]) == list(range(32))
    assert bench.rank_blocks(0, 1, 20, 4) == [0, 1, 2, 3] * 5


def _pinned_digest():
    with open(os.path.join(bench.ROOT, "profiles", "roofline_traffic.txt")) as f:
        for line in f:
            if line.startswith("csrc_sha256:"):
                return line.split(":", 1)[1].strip()
    return None


def test_traffic_records_parse():
    recs = bench.traffic_records()
    assert recs, "profiles/roofline_traffic.txt holds at least one record"
    for r in recs:
        assert {"stage", "precision", "grid_voxels", "dram_bytes_per_system_apply", "csrc_sha256"} <= set(r)


def test_traffic_pin_lookup():
    t = bench.traffic_from_profile(3, "mixed", N128, 8)
    if _pinned_digest() != bench._csrc_digest():
        # the kernels changed since the capture: the bench must not report stale counters
        assert t is None
        return
    # every stage of both precisions is pinned, each within 15% of its algorithmic bytes (no
    # wasted re-reads); the z pass shares the spectrum among the 8 systems of a frequency
    for st in range(6):
        for prec, b, c in (("mixed", 8, 4), ("fp64", 16, 8)):
            v = bench.traffic_from_profile(st, prec, N128, 8)
            assert v is not None and 0.85 < v / bench.stage_bytes(st, N128, b, c, 8) < 1.15, (st, prec)
    assert bench.traffic_from_profile(3, "dfloat", N128, 8) is None
    assert bench.traffic_from_profile(3, "mixed", N128, 2) is None      # another sharing: not pinned
    # scaled to another grid by the number of voxels
    assert abs(bench.traffic_from_profile(3, "mixed", (64, 64, 64), 8) - t / 8) < 1.0
