"""Host-side rules of the benchmark (no GPU): which runs also time the
second window after the kidnap (steps 60-99), and that both arms then build
the same 100-step trajectory; the per-stage bound model's FP64 terms; the
accuracy summary of the representative state."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _args(steps, warmup, after="auto", init="uniform"):
    return argparse.Namespace(steps=steps, warmup=warmup, after_kidnap=after, init=init)


def test_second_window_only_in_benchmark_runs():
    assert bench.times_after_kidnap(_args(40, 10))                 # the default run
    assert not bench.times_after_kidnap(_args(2, 3))               # a profiling run
    assert not bench.times_after_kidnap(_args(40, 10, "off"))
    assert not bench.times_after_kidnap(_args(20, 10, init="tracking"))
    assert not bench.times_after_kidnap(_args(60, 10))             # the first window would cross the kidnap
    assert bench.times_after_kidnap(_args(5, 3, "on"))
    lo, hi = bench.KIDNAP_WINDOW
    assert (lo, hi) == (60, 100)


def test_stage_bounds_take_the_larger_of_bytes_and_flops():
    n, K = 1 << 20, 32
    fp32, fp64_peak = 75.0, 1.2
    b = bench.stage_bounds_ms(n, K, pairs_per_step=8e9, hbm_gbs=6644.1, fp32_tflops=fp32, fp64_tflops=fp64_peak)
    # the posterior: 10 sweeps x (K x 16 + 8) B + 40 B a particle from HBM, against
    # 20K + 2K + 70 FP64 flops a particle at the FP64 peak
    hbm = n * (10 * (K * 16 + 8) + 40) / 6644.1e9 * 1e3
    fp64 = n * (20 * K + 2 * K + 70) / (fp64_peak * 1e12) * 1e3
    assert abs(b["posterior"] - max(hbm, fp64)) < 1e-12
    # the likelihood: one 32-byte sector a pair against 222 flops a pair
    lk = max(8e9 * bench.LK_SECTOR_BYTES_PER_PAIR / 6644.1e9, 8e9 * bench.LK_FLOPS_PER_PAIR / (fp32 * 1e12))
    assert abs(b["likelihood"] - 1e3 * lk) < 1e-9


def test_accuracy_summary():
    """Windows, first localised steps (0.3 m and 3 deg) and the last step."""
    import numpy as np
    d = np.deg2rad
    errs = [(d(10.0), 5.0)] * 12 + [(d(1.0), 0.1)] * 38 + [(d(40.0), 30.0)] * 15 + [(d(2.9), 0.29)] * 35
    a = bench.accuracy_summary(errs, 10, 50, True)
    assert a["first_localised_step"] == 12
    assert a["first_localised_after_kidnap"] == 65
    assert a["window_timed"]["localised_fraction"] == 38 / 40
    assert a["window_after_kidnap"]["localised_fraction"] == 35 / 40
    assert a["last_step"]["step"] == 99 and a["last_step"]["dist_m"] == 0.29
    assert abs(a["last_step"]["angle_deg"] - 2.9) < 1e-12
    b = bench.accuracy_summary(errs[:20], 3, 20, False)
    assert "window_after_kidnap" not in b and b["window_timed"]["steps"] == "3-19"


def test_profile_commands_parse():
    """Every bench command a committed profile summary gives is accepted by
    the bench's own parser (the summaries stay reproducible)."""
    import glob
    import shlex
    cmds = []
    for path in glob.glob(os.path.join(ROOT, "profiles", "*")):
        for line in open(path):
            if "python bench.py" in line:
                tail = line.split("python bench.py", 1)[1]
                tail = tail.split(">")[0].split("&&")[0].replace("\\", " ")
                cmds.append((os.path.basename(path), shlex.split(tail)))
    assert len(cmds) >= 6
    ap = bench.build_parser()
    for name, argv in cmds:
        a = ap.parse_args(argv)
        assert a.warmup >= 3, (name, argv)
