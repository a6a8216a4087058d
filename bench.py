#!/usr/bin/env python
"""Throughput of one MegaParticles filter step on GB300.

A step = prediction (Eq. 1), scan Gaussians, LSH neighbour-list update
(Eq. 9-10, Algorithm 1), likelihood + Gauss-Newton sums (Eq. 2-4), GN solve,
SVGD update (Eq. 5-8) and posterior propagation (Eq. 11), all in the CUDA
library, through its C ABI.

Workload (paper scale, synthetic): 200 x 200 x 20 m outdoor scene with 1M map
points, 2^20 particles uniform over the free space, 8192-point scans from a
32-beam 360-degree sensor along a 1 m/step trajectory, K = 32 neighbours.
Steps 0 .. W+K-1 of the trajectory are run: W untimed, K timed. A second
window, steps 60-99 (after the kidnap at step 50: identity odometry with a
100x covariance and 3 blackout steps), is timed after the first and reported
beside it ("after_kidnap"), when at least 20 steps are timed and the first
window ends by step 60 (not in short profiling runs).

Prints one JSON line. --impl reference times the FP64 CPU oracle instead, on
a bounded sample of the same workload (extrapolated to the full particle
count). Under torchrun every rank runs an independent replica on its own GPU
("replicas only": the filter has no data-path exchange on one GPU per
instance); value = steps of all ranks / max elapsed over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SVGD filter steps/s and particle·point evals/s at 2^20 particles; % GB300 roofline"
N_PARTICLES = 1 << 20
N_POINTS = 8192
N_MAP = 1_000_000
# FP32 operations of one particle x scan-point pair in the likelihood kernel's
# formulation (fused multiply-add = 2): transform 18, voxel 9, lever arm 3,
# residual 3, normal rotation 15, sign and s, d 14, closed-form information
# matrix scalars 14, cost 22, inlier log-likelihood 1, Omega 27, g = Omega e 15,
# [q]x Omega 27, Hessian/gradient accumulation 54.
LK_FLOPS_PER_PAIR = 222
# One random 32-byte NNF sector from DRAM per pair: the HBM bound of the
# likelihood while particles are spread (the 0.5 GB grid does not fit in L2).
LK_SECTOR_BYTES_PER_PAIR = 32
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
ALU_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25          # nominal GB300 FP64 (non-tensor)


def measured_peaks():
    """HBM GB/s and bf16 TFLOP/s measured on this GPU type (MEASURED_PEAKS.json)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def stage_bounds_ms(n, K, pairs_per_step, hbm_gbs):
    """Lower bound of each stage's time per step: max(bytes / HBM peak, flops /
    ALU peak) with the algorithmic bytes and flops of one step (per particle
    unless stated). FP64 stages use the FP64 peak."""
    bw = hbm_gbs * 1e9
    f32 = ALU_PEAK_TFLOPS * 1e12
    f64 = FP64_PEAK_TFLOPS * 1e12
    C = K
    b = {
        # pose in/out (2 x 32 B) + Philox noise
        "predict": (n * 64 / bw, 0.0),
        # 8192 points: brute-force radius kNN (N^2 distances, 8 flops) + normals
        "scan": (N_POINTS * 64 / bw, N_POINTS * N_POINTS * 8 / f32),
        # pose read 32 B + key/id write 8 B; SE(3) log in FP64 (~300 flops)
        "lsh": (n * 40 / bw, n * 300 / f64),
        # 4 radix passes of 8-byte (key, id) read + write, histogram read
        "sort": (n * 4 * 20 / bw, 0.0),
        # old list + window ids, (K + C) 32-byte pose gathers, list/k/d writes
        "merge": (n * (K * 4 + C * 4 + (K + C) * 32 + K * 32) / bw, n * (K + C) * 120 / f32),
        # GN sums 29 x 4 B in, psi 32 B out; FP64 LDL^T of a 6x6 (~250 flops)
        "solve": (n * (29 * 4 + 32) / bw, n * 250 / f64),
        # list ids, k, d (K x 32 B) + K psi gathers (32 B) + pose in/out + phi
        "svgd": (n * (K * 64 + 96) / bw, n * K * 30 / f32),
        # 10 sweeps x K x (id 4 + k 4 + p 8) + normalisation passes (5 x 8 B);
        # FP64: 10 sweeps x K FMAs, the weights (K adds, K multiplies), exp and log
        "posterior": (n * (10 * (K * 16 + 8) + 40) / bw, n * (20 * K + 2 * K + 70) / f64),
    }
    out = {k: 1e3 * max(v) for k, v in b.items()}
    out["likelihood"] = 1e3 * max(pairs_per_step * LK_SECTOR_BYTES_PER_PAIR / bw,
                                  pairs_per_step * LK_FLOPS_PER_PAIR / f32)
    return out


def workload_desc(nvalid=None):
    d = {"workload": "outdoor 200x200x20 m, 2^20 particles x 8192-point scans, 1M map points, K=32",
         "particles": N_PARTICLES, "scan_points": N_POINTS, "map_points": N_MAP, "K": 32,
         "nnf_res_m": 0.2, "l2": "working set larger than L2 (NNF grid ~0.5 GB, neighbour lists ~1.2 GB): no flush"}
    if nvalid is not None:
        d["scan_points_valid_mean"] = nvalid
    return d


KIDNAP_WINDOW = (60, 100)   # the second timed window: steps 60-99, after the kidnap at step 50


def times_after_kidnap(args):
    """Whether the GPU arm times the second window (steps 60-99); both arms
    then build the 100-step trajectory, so they run the same scene."""
    n_steps = args.warmup + args.steps
    return args.after_kidnap == "on" or (args.after_kidnap == "auto" and args.steps >= 20
                                         and n_steps <= KIDNAP_WINDOW[0] and args.init == "uniform")


def make_workload(n_steps, n_particles=None, init="uniform"):
    """The outdoor trajectory workload. init="tracking" replaces the uniform
    particles by a cloud around the first ground-truth pose (0.5 m, 0.05 rad):
    the converged regime of the filter."""
    from paper_2404_16370_gb300 import synth
    wl = synth.outdoor_workload(n_particles=n_particles or N_PARTICLES, n_steps=max(n_steps, 1), n_map=N_MAP,
                                n_points=N_POINTS)
    if init == "tracking":
        wl.particles = synth.tracking_particles(wl.gt[0], len(wl.particles), seed=14)
    return wl


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if "Active" in v and "Not" not in v})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def rank_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device):
    """Largest value over the ranks (timing: the slowest rank defines the job)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps, world, t_max):
    """Whole-job throughput: steps of all ranks / elapsed time of the slowest rank."""
    return steps * world / t_max


def traffic_from_profile():
    """DRAM bytes per likelihood launch from the committed ncu summary, or None
    when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "k_likelihood_outdoor.txt")
    src = os.path.join(ROOT, "paper_2404_16370_gb300", "csrc", "k_likelihood.cu")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_md5") != hashlib.md5(open(src, "rb").read()).hexdigest():
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_setup(wl, n_sample):
    from oracle import oracle as O
    P = O.Params.outdoor(N_PARTICLES)
    t = time.perf_counter()
    om = O.OracleMap(wl.map_points, P)
    init_s = time.perf_counter() - t
    f = O.OracleFilter(om, P, wl.particles[:n_sample].copy())
    return O, f, init_s


def oracle_step_time(f, wl, s):
    t = time.perf_counter()
    f.step(wl.scans[s], wl.odom[s], wl.odom_cov[s])
    return time.perf_counter() - t


def cpu_baseline(wl, n_sample=4096):
    O, f, _ = oracle_setup(wl, n_sample)
    dt = oracle_step_time(f, wl, 0)
    cores = os.cpu_count()
    steps_s = 1.0 / (dt * N_PARTICLES / n_sample)
    return {"value": steps_s, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": f"one FP64 oracle step on {n_sample} of the 2^20 particles (full 8192-point scan, full 1M-point "
                      f"map; {dt:.2f} s), extrapolated linearly to 2^20 particles"}


def run_reference(args):
    world, rank, _ = dist_setup("gloo")
    if rank != 0:
        return
    n_sample = args.sample
    n_steps = args.warmup + args.steps
    wl = make_workload(max(n_steps, KIDNAP_WINDOW[1]) if times_after_kidnap(args) else n_steps)
    O, f, init_s = oracle_setup(wl, n_sample)
    for s in range(args.warmup):
        oracle_step_time(f, wl, s)
    times = [oracle_step_time(f, wl, args.warmup + k) for k in range(args.steps)]
    dt = float(np.mean(times))
    value = 1.0 / (dt * N_PARTICLES / n_sample)
    sample = (f"{n_sample} of the 2^20 particles per step (full scan and map), {dt:.2f} s per sampled step, "
              f"extrapolated linearly to 2^20 particles")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_desc(),
           "cpu_baseline": {"value": value, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def random_read_probe(torch, mp, n_words, stream):
    """Context for the sector roofline: the rate of independent, uniformly
    random 4-byte reads over a buffer the size of the NNF grid (each fetches
    one 32-byte DRAM sector), outside the timed region. The likelihood's
    lookups are not uniform (consecutive points of a particle fall in nearby
    voxels, often in the same DRAM row), so this is a reference below it, not a
    ceiling; the roofline's peak stays the measured copy bandwidth."""
    try:
        words = torch.zeros(int(n_words), dtype=torch.int32, device=torch.cuda.current_device())
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        blocks, reads = 8 * sms, 256
        ms = mp.mp_probe_random_reads(words, blocks, reads, repeats=5, cuda_stream=stream.cuda_stream)
        n_reads = blocks * 256 * reads
        del words
        return {"buffer_bytes": 4 * int(n_words), "reads_per_run": n_reads, "ms_per_run": ms,
                "reads_per_s": n_reads / (ms / 1e3), "sector_gbs": n_reads * 32 / (ms / 1e3) / 1e9,
                "method": "mp_probe_random_reads: independent LCG indices, 8 CTAs of 256 threads per SM"}
    except Exception as e:   # a measurement aid only
        return {"error": str(e)}


def run_gpu(args):
    import torch
    world, rank, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    from paper_2404_16370_gb300 import mp

    n_steps = args.warmup + args.steps
    after_kidnap = times_after_kidnap(args)
    wl = make_workload(max(n_steps, KIDNAP_WINDOW[1]) if after_kidnap else n_steps, init=args.init)
    stream = torch.cuda.Stream()
    params = mp.mp_default_params(mp.MP_PRESET_OUTDOOR, N_PARTICLES)
    params.seed = 4 + rank
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = mp.mp_init_map(wl.map_points, params, cuda_stream=stream.cuda_stream)
    init_map_s = time.perf_counter() - t0
    mp.mp_set_precision(ctx, {"fp32": mp.MP_PREC_FP32, "bf16": mp.MP_PREC_BF16, "fp16": mp.MP_PREC_FP16}[args.precision])
    scans_dev = [torch.from_numpy(s).to(f"cuda:{local}") for s in wl.scans]
    scans_pin = [torch.from_numpy(s).pin_memory() for s in wl.scans]
    torch.cuda.synchronize()

    def run_steps(lo, hi, host=False):
        for s in range(lo, hi):
            sc = scans_pin[s] if host else scans_dev[s]
            mp.mp_step(ctx, sc if len(sc) else None, wl.odom[s], wl.odom_cov[s])
            if host:
                mp.mp_get_posterior(ctx)          # D2H of the step's result (best pose, its probability)

    def barrier():
        rank_barrier(world)

    def max_over_ranks(x):
        return reduce_max(x, world, f"cuda:{local}")

    try:
        # ---- device-resident inputs: the timed steps W .. W+K-1
        mp.mp_init_particles(ctx, N_PARTICLES, poses=wl.particles)
        run_steps(0, args.warmup)
        torch.cuda.synchronize()
        mp.mp_set_timing(ctx, True)
        launches0 = mp.mp_kernel_launches(ctx)
        gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local] \
            if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local)
        clocks = ClockSampler(gpu_index)
        time.sleep(0.25)
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        run_steps(args.warmup, n_steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        launches = mp.mp_kernel_launches(ctx) - launches0
        stage_ms, stage_runs, pairs = mp.mp_stage_times(ctx)
        mp.mp_set_timing(ctx, False)
        best, best_p = mp.mp_get_posterior(ctx)
        t_max = max_over_ranks(elapsed)
        after = None
        if after_kidnap and n_steps <= KIDNAP_WINDOW[0]:
            # ---- second window: steps 60-99, after the kidnap (run on from the first window)
            lo, hi = KIDNAP_WINDOW
            run_steps(n_steps, lo)
            torch.cuda.synchronize()
            barrier()
            ev0.record(stream)
            run_steps(lo, hi)
            ev1.record(stream)
            torch.cuda.synchronize()
            t_after = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
            _, best_p_after = mp.mp_get_posterior(ctx)
            after = {"steps": f"{lo}-{hi - 1}", "value": (hi - lo) * world / t_after, "unit": "steps/s",
                     "ms_per_step": 1e3 * t_after / (hi - lo), "best_prob_last_step": best_p_after,
                     "note": "kidnap at step 50 (identity odometry, 100x covariance, 3 blackout steps)"}

        # ---- end to end through host (pinned) buffers: same steps again
        mp.mp_init_particles(ctx, N_PARTICLES, poses=wl.particles)
        run_steps(0, args.warmup, host=True)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        run_steps(args.warmup, n_steps, host=True)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
        nnf_voxels = int(np.prod(mp.mp_map_info(ctx)["dims"].astype(np.int64)))
    finally:
        mp.mp_destroy(ctx)
    probe = random_read_probe(torch, mp, nnf_voxels, stream) if rank == 0 else None

    if rank != 0:
        return
    steps_total = args.steps * world
    value = job_value(args.steps, world, t_max)
    pairs_rank = pairs
    lk_ms = stage_ms["likelihood"]
    lk_runs = max(stage_runs["likelihood"], 1)
    lk_flops = LK_FLOPS_PER_PAIR * pairs_rank
    achieved = lk_flops / (lk_ms / 1e3) / 1e12 if lk_ms > 0 else None
    traffic = traffic_from_profile() if args.precision == "fp32" else None
    n_timed_scans = [len(wl.scans[s]) for s in range(args.warmup, n_steps)]
    h2d = int(np.mean([n * 12 for n in n_timed_scans])) + 16 * 8 + 36 * 8
    d2h = 7 * 4 + 8
    nvalid_mean = pairs_rank / N_PARTICLES / max(lk_runs, 1)
    hbm_gbs, hbm_src = measured_peaks()
    pairs_step = pairs_rank / lk_runs
    lk_s = lk_ms / 1e3 / lk_runs
    sector_gbs = pairs_step * LK_SECTOR_BYTES_PER_PAIR / lk_s / 1e9 if lk_s > 0 else None
    stage_meas = {k: v / max(stage_runs[k], 1) for k, v in stage_ms.items()}
    bounds = stage_bounds_ms(N_PARTICLES, 32, pairs_step, hbm_gbs)
    step_bound = sum(bounds.values())
    out = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16+f32", "fp16": "f16+f32"}[args.precision],
        "data": "synthetic",
        "config": {**workload_desc(round(nvalid_mean, 1)), "init": args.init, "precision": args.precision},
        "pair_evals_per_s": pairs_rank * world / t_max,
        "roofline": {"bound": "alu", "kernel": "k_likelihood", "achieved": achieved, "peak": ALU_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": (achieved / ALU_PEAK_TFLOPS) if achieved else None,
                     "traffic": traffic,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz max SM clock",
                     "flops_per_pair": LK_FLOPS_PER_PAIR, "pairs_per_launch": pairs_rank / lk_runs,
                     "avg_launch_ms": lk_ms / lk_runs},
        "roofline_hbm_sector": {"bound": "hbm", "kernel": "k_likelihood", "achieved": sector_gbs, "peak": hbm_gbs,
                                "unit": "GB/s", "frac": (sector_gbs / hbm_gbs) if sector_gbs else None,
                                "peak_source": hbm_src,
                                "model": "one 32-byte NNF sector from DRAM per pair (spread particles)",
                                "uniform_random_reads": probe},
        "roofline_step": {"bound_ms": step_bound, "measured_ms": 1e3 * t_max / args.steps,
                          "frac": step_bound / (1e3 * t_max / args.steps),
                          "stage_bound_ms": bounds,
                          "model": "sum over stages of max(algorithmic bytes / HBM peak, flops / ALU peak)"},
        "stage_ms_per_step": stage_meas,
        "e2e": {"value": steps_total / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "after_kidnap": after,
        "gpu_launches": launches,
        "clocks": clk,
        "init_map_s": round(init_map_s, 3),
        "best_prob_last_step": best_p,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_sample)
    print(json.dumps(out), flush=True)


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--sample", type=int, default=1024, help="particles per step in the reference arm's sample")
    ap.add_argument("--cpu-sample", type=int, default=4096, help="particles in the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--init", default="uniform", choices=["uniform", "tracking"],
                    help="particles uniform over the map (the benchmark) or around the true pose")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="arithmetic of the likelihood stage (16-bit per-pair arithmetic, FP32 sums)")
    ap.add_argument("--after-kidnap", default="auto", choices=["auto", "on", "off"],
                    help="also time steps 60-99 (after the kidnap at step 50); auto: when >= 20 steps are timed")
    ap.add_argument("--particles", type=int, default=N_PARTICLES,
                    help="particle count (profiling runs of a smaller case; the benchmark is 2^20)")
    return ap


def main():
    global N_PARTICLES
    ap = build_parser()
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    N_PARTICLES = args.particles
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
