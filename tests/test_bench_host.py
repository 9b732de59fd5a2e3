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


def _pinned_digest():
    with open(os.path.join(bench.ROOT, "profiles", "roofline_traffic.txt")) as f:
        for line in f:
            if line.startswith("csrc_sha256:"):
                return line.split(":", 1)[1].strip()
    return None


def test_traffic_pin_lookup():
    t = bench.traffic_from_profile(3, "mixed", N128)
    if _pinned_digest() != bench._csrc_digest():
        # the kernels changed since the capture: the bench must not report stale counters
        assert t is None
        return
    # the FP32 z pass reads and writes a little less than its algorithmic bytes (the spectrum is
    # shared by the two systems of the capture): no wasted re-reads
    assert t is not None and 0.9 < t / bench.stage_bytes(3, N128, 8, 4) < 1.0
    assert bench.traffic_from_profile(3, "fp64", N128) is None
    assert bench.traffic_from_profile(2, "mixed", N128) is None
    # scaled to another grid by the number of voxels
    assert abs(bench.traffic_from_profile(3, "mixed", (64, 64, 64)) - t / 8) < 1.0
