"""Learned proposal for the box room: data generation with the GPU sensor
simulator, training of the PointNet-style mixture network with its own
kernels, particle seeding from the mixture and the comparison with uniform
seeding on seeded localisation trials.

    python -m paper_2404_16370_gb300.proposal --samples 200000 --epochs 8 --trials 500

trains a network (pose/scan pairs ray-cast from the box room), then runs the
trials of paper_2404_16370_gb300.localise twice, with uniform particles and
with 90% of the particles drawn from the mixture of each trial's scan (10%
uniform), and prints one JSON line per seeding.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
from scipy.spatial.transform import Rotation

from . import localise, mp, synth

N_POINTS = 1024
IN_SCALE = 5.0
# pose target (x, y, z, yaw, pitch, roll) = value * scale + offset in the box room
SCALE = np.array([5.0, 5.0, 0.75, 1.0, 0.1, 0.1], np.float32)
OFFSET = np.array([0.0, 0.0, 1.25, 0.0, 0.0, 0.0], np.float32)


def room_boxes(room) -> np.ndarray:
    b = room.boxes
    return np.concatenate([b.c, b.z0[:, None], b.size, b.yaw[:, None]], 1).astype(np.float32)


def sample_poses(room, n, seed):
    """n poses as box_room_gt_pose draws them: free positions 0.5 m from every
    surface, z in [0.5, 2], yaw uniform, pitch and roll within 5 degrees."""
    rng = np.random.default_rng(seed)
    out = np.zeros((0, 3))
    while len(out) < n:
        xyz = np.stack([rng.uniform(-room.half + 1, room.half - 1, 2 * n), rng.uniform(-room.half + 1, room.half - 1, 2 * n),
                        rng.uniform(0.5, 2.0, 2 * n)], -1)
        out = np.concatenate([out, xyz[room.free(xyz, margin=0.5)]])
    xyz = out[:n]
    yaw = rng.uniform(-np.pi, np.pi, n)
    pitch, roll = np.deg2rad(rng.uniform(-5, 5, (2, n)))
    return synth.poses_from_euler(xyz, yaw, pitch, roll)


def targets_of(poses) -> np.ndarray:
    """Normalised (x, y, z, yaw, pitch, roll) of (n, 7) poses."""
    ypr = Rotation.from_quat(np.asarray(poses[:, :4], np.float64)).as_euler("ZYX")
    v = np.concatenate([poses[:, 4:7], ypr], 1)
    return ((v - OFFSET) / SCALE).astype(np.float32)


class BoxRoomSim:
    """GPU ray-casting of box-room scans along the 1024 Fibonacci directions."""

    def __init__(self, room, device="cuda", n_points=N_POINTS):
        import torch
        self.room = room
        self.boxes = torch.from_numpy(room_boxes(room)).to(device)
        self.dirs = torch.from_numpy(synth.fibonacci_sphere(n_points).astype(np.float32)).to(device)
        self.device = device

    def scans(self, poses, noise, seed, chunk=8192):
        import torch
        poses_t = torch.as_tensor(np.asarray(poses, np.float32)).to(self.device)
        out = torch.empty((len(poses_t), len(self.dirs), 3), device=self.device)
        for k in range(0, len(poses_t), chunk):
            mp.mp_pn_sim_box_room(self.boxes, self.room.half, self.room.height, poses_t[k:k + chunk].contiguous(),
                                  self.dirs, noise, seed + k, out[k:k + chunk])
        return out


class Proposal:
    """The network with its trainer and sampler (one CUDA context stream: torch's current)."""

    def __init__(self, max_batch=128, seed=0):
        self.max_batch = max_batch
        self.net = mp.mp_pn_create(N_POINTS, max_batch, IN_SCALE, SCALE, OFFSET, seed)

    def close(self):
        if self.net is not None:
            mp.mp_pn_destroy(self.net)
            self.net = None

    def train(self, scans, targets, epochs, lr=1e-3, seed=0, log=None):
        """Adam over shuffled mini-batches; returns the mean loss of each epoch."""
        import torch
        n = len(scans)
        B = self.max_batch
        tg = torch.as_tensor(targets).to(scans.device)
        loss = torch.zeros(1, device=scans.device)
        acc = torch.zeros(1, device=scans.device)
        g = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g).to(scans.device)
            acc.zero_()
            nb = 0
            for k in range(0, n - B + 1, B):
                idx = perm[k:k + B]
                xb = scans.index_select(0, idx).contiguous()
                yb = tg.index_select(0, idx).contiguous()
                mp.mp_pn_loss_grad(self.net, xb, yb, loss)
                mp.mp_pn_adam_step(self.net, lr)
                acc += loss
                nb += 1
            hist.append(float(acc.item()) / max(nb, 1))
            if log:
                log(f"epoch {ep}: mean loss {hist[-1]:.4f}")
        return hist

    def mixture(self, scans):
        import torch
        out = torch.empty((len(scans), mp.MP_PN_OUT), device=scans.device)
        for k in range(0, len(scans), self.max_batch):
            mp.mp_pn_forward(self.net, scans[k:k + self.max_batch].contiguous(), out[k:k + self.max_batch])
        return out

    def sample(self, mix, n, seed):
        import torch
        out = torch.empty((n, 7), device=mix.device)
        mp.mp_pn_sample(self.net, mix.contiguous(), n, seed, out)
        return out


def seeding_from(prop, sim, trials, frac=0.9, seed=0):
    """Seeding callback for localise.run: frac of the particles from the mixture
    of the trial's 1024-ray scan, the rest kept from the uniform set (a CUDA
    tensor: the drawn poses never leave the device)."""
    import torch

    def seed_fn(t, _scan, parts):
        gt = trials[t][0]
        sc = sim.scans(gt[None], 0.02, seed + 7919 * (t + 1))
        mix = prop.mixture(sc)
        n_mix = int(round(frac * len(parts)))
        out = torch.from_numpy(np.ascontiguousarray(parts)).to(sc.device)
        out[:n_mix] = prop.sample(mix[0], n_mix, seed + t)
        return out
    return seed_fn


def proposal_quality(prop, sim, trials, n=4096, seed=0):
    """How close the network's proposals come to the truth on the trials: the
    error of the heaviest component's mean, and the fraction of trials with at
    least one of n drawn poses within 0.3 m / 3 degrees (which a uniform set
    of the same size reaches in a few per cent of trials)."""
    import torch
    best_d, best_a, hit = [], [], []
    for t, trial in enumerate(trials):
        gt = trial[0]
        sc = sim.scans(gt[None], 0.02, seed + 7919 * (t + 1))
        mix = prop.mixture(sc)[0]
        c = int(torch.argmax(mix[:32]).item())
        m = mix[32 + 6 * c:38 + 6 * c].cpu().numpy() * SCALE + OFFSET
        g = targets_of(gt[None])[0] * SCALE + OFFSET
        best_d.append(float(np.linalg.norm(m[:3] - g[:3])))
        best_a.append(float(abs((m[3] - g[3] + np.pi) % (2 * np.pi) - np.pi)))
        poses = prop.sample(mix, n, seed + t).cpu().numpy()
        ang = (Rotation.from_quat(poses[:, :4].astype(np.float64)).inv() *
               Rotation.from_quat(np.asarray(gt[:4], np.float64))).magnitude()
        dist = np.linalg.norm(poses[:, 4:7] - gt[4:7], axis=1)
        hit.append(bool(np.any((dist <= localise.MAX_DIST) & (ang <= localise.MAX_ANG))))
    return {"heaviest_component_dist_median_m": float(np.median(best_d)),
            "heaviest_component_yaw_err_median_deg": float(np.rad2deg(np.median(best_a))),
            "trials_with_a_draw_within_tolerance": float(np.mean(hit))}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--samples", type=int, default=200_000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--trials", type=int, default=500)
    ap.add_argument("--particles", type=int, default=4096)
    ap.add_argument("--max-steps", type=int, default=30)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--svgd-precond", default="0,1", help="comma list of mp_params.svgd_precond values")
    a = ap.parse_args()
    import torch
    room = synth.box_room(1)
    sim = BoxRoomSim(room)
    t0 = time.perf_counter()
    poses = sample_poses(room, a.samples, seed=1000 + a.seed)
    scans = sim.scans(poses, 0.02, seed=2000 + a.seed)
    targets = targets_of(poses)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    prop = Proposal(a.batch, seed=a.seed)
    try:
        t0 = time.perf_counter()
        hist = prop.train(scans, targets, a.epochs, a.lr, seed=a.seed, log=lambda s: print(s, flush=True))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        del scans
        print(json.dumps({"train_samples": a.samples, "epochs": a.epochs, "batch": a.batch, "data_s": round(t_data, 2),
                          "train_s": round(t_train, 2), "loss_per_epoch": [round(h, 4) for h in hist]}), flush=True)
        if a.trials <= 0:
            return
        _, trials = localise.make_trials(a.trials, a.particles, seed0=100 + a.seed)
        print(json.dumps({"proposal_quality": proposal_quality(prop, sim, trials, a.particles, seed=a.seed)}),
              flush=True)
        for pre in (int(v) for v in a.svgd_precond.split(",")):
            for name, fn in (("uniform", None), ("learned", seeding_from(prop, sim, trials, seed=a.seed))):
                t0 = time.perf_counter()
                errs = localise.run(room, trials, "fp32", a.max_steps, seeding=fn, svgd_precond=pre)
                res = {"scene": "box_room", "seeding": name, "svgd_precond": pre, "particles": a.particles,
                       "max_steps": a.max_steps, "wall_s": round(time.perf_counter() - t0, 2),
                       **localise.summarise(errs)}
                res.pop("steps_to_localise")
                print(json.dumps(res), flush=True)
    finally:
        prop.close()


if __name__ == "__main__":
    main()
