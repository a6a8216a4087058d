"""Many independent localisation instances stepped together.

Workload: 64 instances on 8 seeded box rooms of 20k map points, particle
counts log-uniform in 2^10..2^13, scans of 512..2048 points (log-uniform).
Each instance keeps one scan (ray-cast from a seeded pose) for every step,
with small odometry and noise. The instances on one map share its device
copy (mp_init_map_shared; --own-maps gives each instance its own).

    python -m paper_2404_16370_gb300.batch --instances 64 --steps 10

times the same steps taken (a) instance by instance with mp_step, one
instance after the other on one stream, and (b) with mp_batch_step (one
CUDA-graph launch per step: every phase one grouped kernel over all
instances, the posterior one persistent cooperative kernel, likelihood
splits picked by timing), and prints one JSON line with instance-steps/s and
particle-point pairs/s of both and how many instances end with a finite,
normalised posterior. All contexts and the batch share one stream: no two
instances' kernels run concurrently.

The mix with outdoor maps of up to 1M points and up to 2^18 particles per
instance is not offered: it stopped with a GPU fault whose cause has not been
found, and stays off the GPU until it is.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import mp, synth


def build_instances(n_inst, seed=0, log2_particles=(10, 13), log2_points=(9, 11)):
    """Box-room instances on 8 seeded rooms (instance i on room i mod 8)."""
    rng = np.random.default_rng(seed)
    maps = [synth.box_room(1 + k) for k in range(8)]
    inst = []
    for i in range(n_inst):
        room = maps[i % len(maps)]
        n_part = int(2 ** rng.uniform(*log2_particles))
        n_pts = int(2 ** rng.uniform(*log2_points))
        gt = synth.box_room_gt_pose(room, 1000 + i)
        scan = synth.scan(room, gt, synth.spherical_dirs(n_pts), 0.02, 2000 + i)
        parts = synth.box_room_particles(n_part, 3000 + i, room.half)
        inst.append(dict(map=i % len(maps), kind="box_room", pts=room.map_points, scan=scan.astype(np.float32),
                         parts=parts, preset=mp.MP_PRESET_BOX_ROOM, n=n_part))
    return inst


def make_contexts(inst, stream, share_maps=True):
    """One context per instance, all on `stream`; with share_maps the
    instances on one map use one device copy of it (mp_init_map_shared)."""
    ctxs, first = [], {}
    for d in inst:
        p = mp.mp_default_params(d["preset"], d["n"])
        if share_maps and d["map"] in first:
            ctx = mp.mp_init_map_shared(first[d["map"]], p, cuda_stream=stream)
        else:
            ctx = mp.mp_init_map(d["pts"], p, cuda_stream=stream)
            first[d["map"]] = ctx
        mp.mp_init_particles(ctx, d["n"], poses=d["parts"])
        ctxs.append(ctx)
    return ctxs


def release(ctxs):
    for c in ctxs:
        mp.mp_destroy(c)


def step_all(ctxs, scans, T, cov, s):
    """mp_step on every instance, one after the other; a failure names the
    instance and the step."""
    for i, c in enumerate(ctxs):
        try:
            mp.mp_step(c, scans[i], T[i], cov[i])
        except mp.MPError as e:
            raise mp.MPError(e.code, f"instance {i}, step {s}: {e}") from None


def odometry(n, step):
    rng = np.random.default_rng(7000 + step)
    T = np.tile(np.eye(4), (n, 1, 1))
    T[:, :3, 3] = rng.normal(0, 0.05, (n, 3))
    cov = np.tile(np.diag([1e-4] * 3 + [2.5e-3] * 3), (n, 1, 1))
    return T, cov


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batched-only", action="store_true", help="time only the batched steps (no mp_step baseline)")
    ap.add_argument("--own-maps", action="store_true",
                    help="one device copy of the map per instance (default: the instances on one map share it)")
    a = ap.parse_args()
    import torch
    t0 = time.perf_counter()
    inst = build_instances(a.instances)
    gen_s = time.perf_counter() - t0
    n = len(inst)
    scans = [d["scan"] for d in inst]
    pairs_step = float(sum(d["n"] * len(d["scan"]) for d in inst))
    res = {"workload": "box-room instances: 2^10..2^13 particles, 512..2048-point scans, 8 rooms of 20k points",
           "device_maps": "one per instance" if a.own_maps else "one per map, shared by its instances",
           "instances": n, "maps": 8, "particles_total": int(sum(d["n"] for d in inst)),
           "scan_points_total": int(sum(len(d["scan"]) for d in inst)), "steps": a.steps, "warmup": a.warmup,
           "inputs_s": round(gen_s, 1)}
    stream = mp.mp_stream_create()
    t_seq = None
    # (a) instance by instance
    if not a.batched_only:
        ctxs = make_contexts(inst, stream, not a.own_maps)
        try:
            for s in range(a.warmup):
                T, cov = odometry(n, s)
                step_all(ctxs, scans, T, cov, s)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in range(a.warmup, a.warmup + a.steps):
                T, cov = odometry(n, s)
                step_all(ctxs, scans, T, cov, s)
            torch.cuda.synchronize()
            t_seq = time.perf_counter() - t0
        finally:
            release(ctxs)
    # (b) batched
    ctxs = make_contexts(inst, stream, not a.own_maps)
    try:
        t0 = time.perf_counter()
        batch = mp.mp_batch_create(ctxs, [len(s) for s in scans], stream, tune_scans=scans)
        create_s = time.perf_counter() - t0
        try:
            for s in range(a.warmup):
                T, cov = odometry(n, s)
                mp.mp_batch_step(batch, scans, T, cov)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in range(a.warmup, a.warmup + a.steps):
                T, cov = odometry(n, s)
                mp.mp_batch_step(batch, scans, T, cov)
            torch.cuda.synchronize()
            t_bat = time.perf_counter() - t0
            splits = [mp.mp_batch_split(batch, i) for i in range(n)]
            # every instance's posterior after the batched steps: finite and normalised
            post_ok = 0
            for c in ctxs:
                mp.mp_get_posterior(c)
                post = mp.mp_get_buffer(c, mp.MP_BUF_POST)
                post_ok += int(bool(np.isfinite(post).all()) and abs(float(post.sum()) - 1.0) < 1e-9)
        finally:
            mp.mp_batch_destroy(batch)
    finally:
        release(ctxs)
        mp.mp_stream_destroy(stream)
    res.update({
        "sequential": None if t_seq is None else {
            "instance_steps_per_s": n * a.steps / t_seq, "pairs_per_s": pairs_step * a.steps / t_seq,
            "ms_per_step": 1e3 * t_seq / a.steps},
        "batched": {"instance_steps_per_s": n * a.steps / t_bat, "pairs_per_s": pairs_step * a.steps / t_bat,
                    "ms_per_step": 1e3 * t_bat / a.steps, "create_s": round(create_s, 2)},
        "speedup": None if t_seq is None else t_seq / t_bat,
        "splits": {str(k): splits.count(k) for k in sorted(set(splits))},
        "posteriors_normalised": f"{post_ok}/{n}",
    })
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
