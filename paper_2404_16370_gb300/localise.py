"""Localisation trials on the 10 x 10 x 3 m box room.

Each trial draws a ground-truth pose (seeded), ray-casts its 512-ray scan
(0.02 m range noise) and runs the filter on that static scan (identity
odometry, no prediction noise) from a fresh particle set for max_steps steps.
A trial localises at the first step whose representative state (the
highest-posterior particle) lies within 0.3 m and 3 degrees of the truth; the
time to localise is that step count. The same trials (poses, scans, initial
particles, LSH draws) are run for every likelihood precision and every
particle seeding, so the forms are compared trial by trial.

    python -m paper_2404_16370_gb300.localise --trials 100 --precision fp32,bf16,fp16

prints one JSON line per (precision, seeding) with the success rate, the
time to localise (median, mean over successes) and the final errors.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import mp, synth

PRECISIONS = {"fp32": mp.MP_PREC_FP32, "bf16": mp.MP_PREC_BF16, "fp16": mp.MP_PREC_FP16}
MAX_DIST, MAX_ANG = 0.3, np.deg2rad(3.0)


def pose_errors(a, b):
    """(rotation angle, translation distance) between two poses (qx qy qz qw tx ty tz)."""
    qa = np.asarray(a[:4], np.float64)
    qb = np.asarray(b[:4], np.float64)
    qa /= np.linalg.norm(qa)
    qb /= np.linalg.norm(qb)
    ang = 2.0 * np.arccos(min(1.0, abs(float(np.dot(qa, qb)))))
    return ang, float(np.linalg.norm(np.asarray(a[4:7], np.float64) - np.asarray(b[4:7], np.float64)))


def make_trials(n_trials, n_particles, seed0=100):
    """Trials (true pose, its scan, the seed and size of the initial particle
    set); the particles are drawn when a trial runs (trial_particles), so that
    large sets are never held for every trial at once."""
    room = synth.box_room(1)
    dirs = synth.spherical_dirs(512)
    trials = []
    for t in range(n_trials):
        gt = synth.box_room_gt_pose(room, seed0 + t)
        sc = synth.scan(room, gt, dirs, 0.02, seed0 + t)
        trials.append((gt, sc, 10_000 + seed0 + t, n_particles))
    return room, trials


def trial_particles(room, trial):
    """The trial's uniform initial particle set (n x 7)."""
    return synth.box_room_particles(trial[3], seed=trial[2], half=room.half)


def run(room, trials, precision, max_steps, seeding=None, stream=None, svgd_precond=0, post_floor=None):
    """Errors (trials, max_steps, 2) of the representative state per step.
    seeding(trial_index, scan, particles) -> particles (numpy or a CUDA
    tensor) replaces the initial set; svgd_precond selects the SVGD reading
    (mp_params.svgd_precond); post_floor (None: the default) the posterior
    floor in nats (mp_params.post_floor; 0: none)."""
    n = trials[0][3]
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, n)
    params.svgd_precond = int(svgd_precond)
    if post_floor is not None:
        params.post_floor = float(post_floor)
    ctx = mp.mp_init_map(room.map_points, params, cuda_stream=stream)
    eye, zero = np.eye(4), np.zeros((6, 6))
    out = np.zeros((len(trials), max_steps, 2))
    try:
        mp.mp_set_precision(ctx, PRECISIONS[precision])
        for t, (gt, sc, _, _) in enumerate(trials):
            parts = trial_particles(room, trials[t])
            p0 = parts if seeding is None else seeding(t, sc, parts)
            mp.mp_init_particles(ctx, n, poses=p0)
            mp.mp_set_step_index(ctx, 0)
            for s in range(max_steps):
                mp.mp_step(ctx, sc, eye, zero)
                best, _ = mp.mp_get_posterior(ctx)
                out[t, s] = pose_errors(best, gt)
    finally:
        mp.mp_destroy(ctx)
    return out


def summarise(errs):
    ok = (errs[:, :, 1] <= MAX_DIST) & (errs[:, :, 0] <= MAX_ANG)
    hit = ok.any(axis=1)
    steps = np.where(hit, ok.argmax(axis=1) + 1, -1)
    return {
        "trials": int(len(errs)),
        "localised": int(hit.sum()),
        "success_rate": float(hit.mean()),
        "time_to_localise_median": float(np.median(steps[hit])) if hit.any() else None,
        "time_to_localise_mean": float(steps[hit].mean()) if hit.any() else None,
        "final_dist_median_m": float(np.median(errs[:, -1, 1])),
        "final_angle_median_deg": float(np.rad2deg(np.median(errs[:, -1, 0]))),
        "final_localised": float(np.mean(ok[:, -1])),
        "steps_to_localise": steps.tolist(),
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--trials", type=int, default=50)
    ap.add_argument("--particles", type=int, default=4096)
    ap.add_argument("--max-steps", type=int, default=30)
    ap.add_argument("--precision", default="fp32,bf16,fp16")
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--svgd-precond", default="0", help="comma list of mp_params.svgd_precond values")
    ap.add_argument("--post-floor", default="700", help="comma list of mp_params.post_floor values (nats; 0: none)")
    a = ap.parse_args()
    room, trials = make_trials(a.trials, a.particles, a.seed)
    for floor in (float(v) for v in a.post_floor.split(",")):
        for pre in (int(v) for v in a.svgd_precond.split(",")):
            for prec in a.precision.split(","):
                t0 = time.perf_counter()
                errs = run(room, trials, prec, a.max_steps, svgd_precond=pre, post_floor=floor)
                res = {"scene": "box_room", "precision": prec, "svgd_precond": pre, "post_floor": floor,
                       "seeding": "uniform", "particles": a.particles, "max_steps": a.max_steps,
                       "wall_s": round(time.perf_counter() - t0, 2), **summarise(errs)}
                res.pop("steps_to_localise")
                print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
