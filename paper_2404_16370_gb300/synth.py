"""Seeded synthetic inputs: scenes, map clouds, a ray-cast range sensor,
particle sets, ground-truth trajectories and odometry.

This module is shared by the CUDA path's tests/benchmarks and by the oracle's
tests. It holds none of the filter's arithmetic (no likelihood, no SE(3) log,
no hashing, no SVGD, no posterior): only scene geometry, ray-primitive
intersection and numpy/scipy random draws (PCG64 via ``numpy.random``, which
is unrelated to the Philox stream the filter itself draws from).

Pose arrays are float32 (n, 7): (qx, qy, qz, qw, tx, ty, tz), sensor-to-world.
Scans are float32 (n, 3) in the sensor frame.

Workloads (shapes of the paper's experiments, Sec. IV-A and IV-B, scaled):
  * box room: 10 x 10 x 3 m room, 8 random boxes (sides 0.3-1.5 m), 20k
    area-uniform map points; 512-ray equal-area spherical scan with N(0, 0.02 m)
    range noise; particles uniform over x, y in [-5, 5], z in [0, 2],
    yaw in [-pi, pi), roll/pitch in [-5, 5] deg.
  * outdoor: 200 x 200 m heightfield (|h| <= 3 m) with 50 box buildings and
    300 poles, 1M area-uniform map points; 32-beam 360 deg sensor
    (elevation -15..15 deg), 0.03 m noise, 10 % dropout, 100 m range, 8192
    returns; particles uniform over the free space at terrain + 1.5 +- 0.5 m;
    a 100-step trajectory at 1 m/step with a kidnap at step 50.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial.transform import Rotation

# ---------------------------------------------------------------------------
# small helpers
# ---------------------------------------------------------------------------


def poses_from_euler(xyz, yaw, pitch, roll) -> np.ndarray:
    """(n,7) float32 poses from positions and Z-Y-X Euler angles."""
    q = Rotation.from_euler("ZYX", np.stack([yaw, pitch, roll], -1)).as_quat()  # (x, y, z, w)
    out = np.concatenate([q, np.asarray(xyz, np.float64)], -1)
    return out.astype(np.float32)


def pose_matrix(pose) -> np.ndarray:
    """4x4 float64 matrix of one (7,) pose."""
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(np.asarray(pose[:4], np.float64)).as_matrix()
    T[:3, 3] = pose[4:7]
    return T


def matrix_pose(T) -> np.ndarray:
    q = Rotation.from_matrix(T[:3, :3]).as_quat()
    return np.concatenate([q, T[:3, 3]]).astype(np.float32)


def fibonacci_sphere(n: int) -> np.ndarray:
    """n equal-area directions on the unit sphere."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.pi * (3.0 - np.sqrt(5.0)) * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], -1)


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------
@dataclass
class Boxes:
    """Yawed boxes: centre (cx, cy), base z0, size (sx, sy, sz), yaw."""
    c: np.ndarray      # (m, 2)
    z0: np.ndarray     # (m,)
    size: np.ndarray   # (m, 3)
    yaw: np.ndarray    # (m,)

    def __len__(self):
        return len(self.yaw)

    def subset(self, keep):
        return Boxes(self.c[keep], self.z0[keep], self.size[keep], self.yaw[keep])

    def ray_hit(self, o, d):
        """Nearest positive hit distance of rays (n,3)/(n,3) with the boxes
        (outside-facing), inf if none."""
        best = np.full(len(o), np.inf)
        for b in range(len(self)):
            cy, sy = np.cos(-self.yaw[b]), np.sin(-self.yaw[b])
            ox = o[:, 0] - self.c[b, 0]
            oy = o[:, 1] - self.c[b, 1]
            lo_ = np.array([-self.size[b, 0] / 2, -self.size[b, 1] / 2, self.z0[b]])
            hi_ = np.array([self.size[b, 0] / 2, self.size[b, 1] / 2, self.z0[b] + self.size[b, 2]])
            lo_o = np.stack([cy * ox - sy * oy, sy * ox + cy * oy, o[:, 2]], -1)
            lo_d = np.stack([cy * d[:, 0] - sy * d[:, 1], sy * d[:, 0] + cy * d[:, 1], d[:, 2]], -1)
            with np.errstate(divide="ignore", invalid="ignore"):
                inv = 1.0 / lo_d
                t1 = (lo_ - lo_o) * inv
                t2 = (hi_ - lo_o) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=1)
            hit = (tmax >= tmin) & (tmin > 1e-6)
            best = np.where(hit & (tmin < best), tmin, best)
        return best

    def contains(self, p, margin=0.0):
        inside = np.zeros(len(p), bool)
        for b in range(len(self)):
            cy, sy = np.cos(-self.yaw[b]), np.sin(-self.yaw[b])
            x = p[:, 0] - self.c[b, 0]
            y = p[:, 1] - self.c[b, 1]
            lx, ly = cy * x - sy * y, sy * x + cy * y
            inside |= ((np.abs(lx) <= self.size[b, 0] / 2 + margin) & (np.abs(ly) <= self.size[b, 1] / 2 + margin)
                       & (p[:, 2] >= self.z0[b] - margin) & (p[:, 2] <= self.z0[b] + self.size[b, 2] + margin))
        return inside

    def footprint(self, xy, margin=0.0):
        inside = np.zeros(len(xy), bool)
        for b in range(len(self)):
            cy, sy = np.cos(-self.yaw[b]), np.sin(-self.yaw[b])
            x = xy[:, 0] - self.c[b, 0]
            y = xy[:, 1] - self.c[b, 1]
            lx, ly = cy * x - sy * y, sy * x + cy * y
            inside |= (np.abs(lx) <= self.size[b, 0] / 2 + margin) & (np.abs(ly) <= self.size[b, 1] / 2 + margin)
        return inside

    def faces(self, top=True, bottom=False):
        """List of (origin, u, v) parallelograms of the box faces."""
        out = []
        for b in range(len(self)):
            R = np.array([[np.cos(self.yaw[b]), -np.sin(self.yaw[b]), 0], [np.sin(self.yaw[b]), np.cos(self.yaw[b]), 0],
                          [0, 0, 1]])
            sx, sy, sz = self.size[b]
            c = np.array([self.c[b, 0], self.c[b, 1], self.z0[b]])
            corners = lambda x, y, z: c + R @ np.array([x, y, z])
            ex, ey, ez = R @ np.array([sx, 0, 0]), R @ np.array([0, sy, 0]), R @ np.array([0, 0, sz])
            out.append((corners(-sx / 2, -sy / 2, 0), ex, ez))
            out.append((corners(-sx / 2, sy / 2, 0), ex, ez))
            out.append((corners(-sx / 2, -sy / 2, 0), ey, ez))
            out.append((corners(sx / 2, -sy / 2, 0), ey, ez))
            if top:
                out.append((corners(-sx / 2, -sy / 2, sz), ex, ey))
            if bottom:
                out.append((corners(-sx / 2, -sy / 2, 0), ex, ey))
        return out


@dataclass
class Cylinders:
    c: np.ndarray    # (m, 2)
    z0: np.ndarray   # (m,)
    r: np.ndarray    # (m,)
    h: np.ndarray    # (m,)

    def __len__(self):
        return len(self.r)

    def subset(self, keep):
        return Cylinders(self.c[keep], self.z0[keep], self.r[keep], self.h[keep])

    def ray_hit(self, o, d):
        best = np.full(len(o), np.inf)
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        for k in range(len(self)):
            ox = o[:, 0] - self.c[k, 0]
            oy = o[:, 1] - self.c[k, 1]
            bq = 2 * (ox * d[:, 0] + oy * d[:, 1])
            cq = ox ** 2 + oy ** 2 - self.r[k] ** 2
            disc = bq * bq - 4 * a * cq
            ok = (disc >= 0) & (a > 1e-12)
            sq = np.sqrt(np.where(ok, disc, 0))
            with np.errstate(divide="ignore", invalid="ignore"):
                t = (-bq - sq) / (2 * a)
            z = o[:, 2] + t * d[:, 2]
            hit = ok & (t > 1e-6) & (z >= self.z0[k]) & (z <= self.z0[k] + self.h[k])
            best = np.where(hit & (t < best), t, best)
            # top cap
            with np.errstate(divide="ignore", invalid="ignore"):
                tc = (self.z0[k] + self.h[k] - o[:, 2]) / d[:, 2]
            px = ox + tc * d[:, 0]
            py = oy + tc * d[:, 1]
            hitc = (tc > 1e-6) & (px * px + py * py <= self.r[k] ** 2)
            best = np.where(hitc & (tc < best), tc, best)
        return best

    def contains(self, p, margin=0.0):
        inside = np.zeros(len(p), bool)
        if len(self) == 0:
            return inside
        from scipy.spatial import cKDTree
        rmax = float(self.r.max()) + margin
        for k, cand in enumerate(cKDTree(p[:, :2]).query_ball_point(self.c, rmax)):
            if not cand:
                continue
            cand = np.asarray(cand)
            q = p[cand]
            dx = q[:, 0] - self.c[k, 0]
            dy = q[:, 1] - self.c[k, 1]
            hit = ((dx * dx + dy * dy <= (self.r[k] + margin) ** 2) & (q[:, 2] >= self.z0[k] - margin)
                   & (q[:, 2] <= self.z0[k] + self.h[k] + margin))
            inside[cand[hit]] = True
        return inside


def _sample_faces(rng, faces, n):
    areas = np.array([np.linalg.norm(np.cross(u, v)) for (_, u, v) in faces])
    counts = rng.multinomial(n, areas / areas.sum())
    pts = []
    for (o, u, v), m in zip(faces, counts):
        if m == 0:
            continue
        a = rng.random((m, 1))
        b = rng.random((m, 1))
        pts.append(o + a * u + b * v)
    return np.concatenate(pts) if pts else np.zeros((0, 3))


# ---------------------------------------------------------------------------
# box room
# ---------------------------------------------------------------------------
@dataclass
class BoxRoom:
    half: float
    height: float
    boxes: Boxes
    map_points: np.ndarray   # (n, 3) float32

    @property
    def kind(self):
        return "box_room"

    def raycast(self, o, d, max_range=np.inf):
        """Distances along rays (world frame); the room is seen from inside."""
        with np.errstate(divide="ignore", invalid="ignore"):
            lo = np.array([-self.half, -self.half, 0.0])
            hi = np.array([self.half, self.half, self.height])
            t_hi = (hi - o) / d
            t_lo = (lo - o) / d
            tx = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
        t_room = np.min(tx, axis=1)
        t = np.minimum(t_room, self.boxes.ray_hit(o, d))
        return np.where(t <= max_range, t, np.inf)

    def free(self, p, margin=0.3):
        ok = (np.abs(p[:, 0]) < self.half - margin) & (np.abs(p[:, 1]) < self.half - margin)
        ok &= (p[:, 2] > margin) & (p[:, 2] < self.height - margin)
        return ok & ~self.boxes.contains(p, margin)


def box_room(seed: int = 1, n_map: int = 20000, n_boxes: int = 8, half: float = 5.0, height: float = 3.0) -> BoxRoom:
    rng = np.random.default_rng(seed)
    size = rng.uniform(0.3, 1.5, (n_boxes, 3))
    c = rng.uniform(-half + 1.0, half - 1.0, (n_boxes, 2))
    yaw = rng.uniform(-np.pi, np.pi, n_boxes)
    boxes = Boxes(c, np.zeros(n_boxes), size, yaw)
    faces = [
        (np.array([-half, -half, 0.0]), np.array([2 * half, 0, 0]), np.array([0, 2 * half, 0])),          # floor
        (np.array([-half, -half, height]), np.array([2 * half, 0, 0]), np.array([0, 2 * half, 0])),       # ceiling
        (np.array([-half, -half, 0.0]), np.array([2 * half, 0, 0]), np.array([0, 0, height])),
        (np.array([-half, half, 0.0]), np.array([2 * half, 0, 0]), np.array([0, 0, height])),
        (np.array([-half, -half, 0.0]), np.array([0, 2 * half, 0]), np.array([0, 0, height])),
        (np.array([half, -half, 0.0]), np.array([0, 2 * half, 0]), np.array([0, 0, height])),
    ] + boxes.faces(top=True)
    pts = np.zeros((0, 3))
    while len(pts) < n_map:
        cand = _sample_faces(rng, faces, n_map)
        hidden = (np.abs(cand[:, 2]) < 1e-9) & boxes.footprint(cand[:, :2])
        hidden |= boxes.contains(cand, margin=-1e-6)
        pts = np.concatenate([pts, cand[~hidden]])
    return BoxRoom(half, height, boxes, pts[:n_map].astype(np.float32))


def box_room_gt_pose(room: BoxRoom, seed: int = 2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    while True:
        xyz = np.array([rng.uniform(-room.half + 1, room.half - 1), rng.uniform(-room.half + 1, room.half - 1),
                        rng.uniform(0.5, 2.0)])
        if room.free(xyz[None], margin=0.5)[0]:
            break
    yaw = rng.uniform(-np.pi, np.pi)
    pitch, roll = np.deg2rad(rng.uniform(-5, 5, 2))
    return poses_from_euler(xyz[None], np.array([yaw]), np.array([pitch]), np.array([roll]))[0]


def box_room_particles(n: int = 4096, seed: int = 3, half: float = 5.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    xyz = np.stack([rng.uniform(-half, half, n), rng.uniform(-half, half, n), rng.uniform(0, 2, n)], -1)
    yaw = rng.uniform(-np.pi, np.pi, n)
    pitch = np.deg2rad(rng.uniform(-5, 5, n))
    roll = np.deg2rad(rng.uniform(-5, 5, n))
    return poses_from_euler(xyz, yaw, pitch, roll)


# ---------------------------------------------------------------------------
# outdoor scene
# ---------------------------------------------------------------------------
@dataclass
class Outdoor:
    half: float
    terms: np.ndarray      # (m, 4): amplitude, kx, ky, phase
    boxes: Boxes
    poles: Cylinders
    map_points: np.ndarray

    @property
    def kind(self):
        return "outdoor"

    def height(self, x, y):
        h = np.zeros(np.broadcast(x, y).shape)
        for a, kx, ky, ph in self.terms:
            h = h + a * np.sin(kx * x + ky * y + ph)
        return h

    def grad(self, x, y):
        gx = np.zeros(np.broadcast(x, y).shape)
        gy = np.zeros_like(gx)
        for a, kx, ky, ph in self.terms:
            cc = a * np.cos(kx * x + ky * y + ph)
            gx = gx + kx * cc
            gy = gy + ky * cc
        return gx, gy

    def raycast(self, o, d, max_range=100.0, step=0.5):
        n = len(o)
        t_ter = np.full(n, np.inf)
        prev = np.zeros(n)
        active = np.ones(n, bool)
        t = 0.0
        above_prev = o[:, 2] - self.height(o[:, 0], o[:, 1]) > 0
        while t < max_range and active.any():
            t_next = min(t + step, max_range)
            p = o + t_next * d
            above = p[:, 2] - self.height(p[:, 0], p[:, 1]) > 0
            crossed = active & above_prev & ~above
            if crossed.any():
                idx = np.nonzero(crossed)[0]
                a = np.full(len(idx), t)
                b = np.full(len(idx), t_next)
                for _ in range(30):
                    m = 0.5 * (a + b)
                    pm = o[idx] + m[:, None] * d[idx]
                    ab = pm[:, 2] - self.height(pm[:, 0], pm[:, 1]) > 0
                    a = np.where(ab, m, a)
                    b = np.where(ab, b, m)
                t_ter[idx] = 0.5 * (a + b)
                active[idx] = False
            above_prev = above
            t = t_next
        tt = np.minimum(t_ter, np.minimum(self.boxes.ray_hit(o, d), self.poles.ray_hit(o, d)))
        return np.where(tt <= max_range, tt, np.inf)

    def solid(self, p, margin=0.0):
        return self.boxes.contains(p, margin) | self.poles.contains(p, margin)


def outdoor(seed: int = 11, n_map: int = 1_000_000, half: float = 100.0, n_boxes: int = 50, n_poles: int = 300,
            clear_path=None) -> Outdoor:
    rng = np.random.default_rng(seed)
    m = 6
    amp = rng.uniform(0.2, 0.5, m)
    wl = rng.uniform(25.0, 120.0, m)
    ang = rng.uniform(0, np.pi, m)
    terms = np.stack([amp, 2 * np.pi / wl * np.cos(ang), 2 * np.pi / wl * np.sin(ang), rng.uniform(0, 2 * np.pi, m)], -1)
    scene = Outdoor(half, terms, None, None, None)
    size = np.stack([rng.uniform(5, 20, n_boxes), rng.uniform(5, 20, n_boxes), rng.uniform(3, 15, n_boxes)], -1)
    bc = rng.uniform(-half + 10, half - 10, (n_boxes, 2))
    byaw = rng.uniform(-np.pi, np.pi, n_boxes)
    bz = scene.height(bc[:, 0], bc[:, 1]) - 3.0
    size[:, 2] += 3.0
    boxes = Boxes(bc, bz, size, byaw)
    pc = rng.uniform(-half + 2, half - 2, (n_poles, 2))
    pr = rng.uniform(0.1, 0.3, n_poles)
    ph = rng.uniform(3, 8, n_poles) + 1.0
    pz = scene.height(pc[:, 0], pc[:, 1]) - 1.0
    poles = Cylinders(pc, pz, pr, ph)
    if clear_path is not None:
        path = np.asarray(clear_path)[:, :2]
        keepb = np.array([np.min(np.linalg.norm(path - bc[b], axis=1)) > 0.75 * np.hypot(*size[b, :2]) + 4.0
                          for b in range(n_boxes)])
        keepp = np.array([np.min(np.linalg.norm(path - pc[k], axis=1)) > 3.0 for k in range(n_poles)])
        boxes = boxes.subset(keepb)
        poles = poles.subset(keepp)
    scene.boxes, scene.poles = boxes, poles
    # area budget: terrain (slope-weighted), building sides + tops, pole sides + tops
    faces = boxes.faces(top=True)
    face_area = sum(np.linalg.norm(np.cross(u, v)) for (_, u, v) in faces)
    pole_area = float(np.sum(2 * np.pi * poles.r * poles.h + np.pi * poles.r ** 2))
    ter_area = (2 * half) ** 2 * 1.02
    tot = face_area + pole_area + ter_area
    n_face = int(n_map * face_area / tot)
    n_pole = int(n_map * pole_area / tot)
    n_ter = n_map - n_face - n_pole
    # terrain: rejection on the slope factor, outside building / pole footprints
    gmax = np.sqrt(1 + (np.sum(np.abs(terms[:, 0]) * np.hypot(terms[:, 1], terms[:, 2]))) ** 2)
    ter = np.zeros((0, 3))
    while len(ter) < n_ter:
        xy = rng.uniform(-half, half, (2 * n_ter, 2))
        gx, gy = scene.grad(xy[:, 0], xy[:, 1])
        acc = rng.random(len(xy)) * gmax < np.sqrt(1 + gx * gx + gy * gy)
        xy = xy[acc]
        z = scene.height(xy[:, 0], xy[:, 1])
        p = np.concatenate([xy, z[:, None]], -1)
        p = p[~boxes.footprint(xy) & ~poles.contains(p)]
        ter = np.concatenate([ter, p])
    ter = ter[:n_ter]
    # building faces above the terrain
    fp = np.zeros((0, 3))
    while len(fp) < n_face:
        cand = _sample_faces(rng, faces, max(n_face, 1))
        cand = cand[cand[:, 2] > scene.height(cand[:, 0], cand[:, 1])]
        fp = np.concatenate([fp, cand])
    fp = fp[:n_face]
    # poles: lateral surface + top disk
    side = 2 * np.pi * poles.r * poles.h
    top = np.pi * poles.r ** 2
    w = np.concatenate([side, top])
    pick = rng.choice(len(w), size=n_pole, p=w / w.sum())
    pp = np.zeros((n_pole, 3))
    is_side = pick < len(poles)
    k = np.where(is_side, pick, pick - len(poles))
    th = rng.uniform(0, 2 * np.pi, n_pole)
    rr = np.where(is_side, poles.r[k], poles.r[k] * np.sqrt(rng.random(n_pole)))
    pp[:, 0] = poles.c[k, 0] + rr * np.cos(th)
    pp[:, 1] = poles.c[k, 1] + rr * np.sin(th)
    pp[:, 2] = np.where(is_side, poles.z0[k] + rng.random(n_pole) * poles.h[k], poles.z0[k] + poles.h[k])
    pts = np.concatenate([ter, fp, pp])
    pts = pts[rng.permutation(len(pts))]
    scene.map_points = pts.astype(np.float32)
    return scene


def outdoor_trajectory(n_steps: int = 100, kidnap_at: int = 50, radius: float = 60.0, seed: int = 12,
                       scene: Outdoor | None = None):
    """Ground-truth poses along two circular arcs at 1 m/step; at `kidnap_at`
    the sensor jumps to a far point of a second arc. Returns (n_steps, 7)."""
    rng = np.random.default_rng(seed)
    a0 = rng.uniform(0, 2 * np.pi)
    a1 = a0 + np.pi + rng.uniform(-0.5, 0.5)
    r1 = radius * 0.5
    xyz, yaw = [], []
    for s in range(n_steps):
        if s < kidnap_at:
            a = a0 + s / radius
            xyz.append([radius * np.cos(a), radius * np.sin(a), 0.0])
            yaw.append(a + np.pi / 2)
        else:
            a = a1 + (s - kidnap_at) / r1
            xyz.append([r1 * np.cos(a) + 10.0, r1 * np.sin(a) - 5.0, 0.0])
            yaw.append(a + np.pi / 2)
    xyz = np.array(xyz)
    if scene is not None:
        xyz[:, 2] = scene.height(xyz[:, 0], xyz[:, 1]) + 1.5
    else:
        xyz[:, 2] = 1.5
    yaw = np.array(yaw)
    return poses_from_euler(xyz, yaw, np.zeros(n_steps), np.zeros(n_steps))


def outdoor_particles(scene: Outdoor, n: int = 1 << 20, seed: int = 13) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = []
    have = 0
    while have < n:
        m = int((n - have) * 1.3) + 64
        xy = rng.uniform(-scene.half, scene.half, (m, 2))
        z = scene.height(xy[:, 0], xy[:, 1]) + 1.5 + rng.uniform(-0.5, 0.5, m)
        p = np.concatenate([xy, z[:, None]], -1)
        p = p[~scene.solid(p, margin=0.2)]
        out.append(p)
        have += len(p)
    xyz = np.concatenate(out)[:n]
    yaw = rng.uniform(-np.pi, np.pi, n)
    pitch = np.deg2rad(rng.uniform(-5, 5, n))
    roll = np.deg2rad(rng.uniform(-5, 5, n))
    return poses_from_euler(xyz, yaw, pitch, roll)


def tracking_particles(center, n: int, seed: int = 14, sigma_t: float = 0.5, sigma_r: float = 0.05) -> np.ndarray:
    """n poses scattered around `center` (tangent noise: sigma_r rad, sigma_t m)."""
    rng = np.random.default_rng(seed)
    rot = Rotation.from_quat(np.asarray(center[:4], np.float64)) * Rotation.from_rotvec(rng.normal(size=(n, 3)) * sigma_r)
    xyz = np.asarray(center[4:7], np.float64) + rng.normal(size=(n, 3)) * sigma_t
    return np.concatenate([rot.as_quat(), xyz], 1).astype(np.float32)


# ---------------------------------------------------------------------------
# sensors
# ---------------------------------------------------------------------------
def spherical_dirs(n: int = 512) -> np.ndarray:
    return fibonacci_sphere(n)


def lidar_dirs(n_beams: int = 32, n_azimuth: int = 512, elev_deg=(-15.0, 15.0)) -> np.ndarray:
    el = np.deg2rad(np.linspace(elev_deg[0], elev_deg[1], n_beams))
    az = np.linspace(-np.pi, np.pi, n_azimuth, endpoint=False)
    E, A = np.meshgrid(el, az, indexing="ij")
    return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)


def scan(scene, pose, dirs, noise: float, seed: int, dropout: float = 0.0, max_range: float = np.inf,
         n_keep: int | None = None) -> np.ndarray:
    """Ray-cast a scan from `pose` (sensor-to-world) along sensor-frame `dirs`.
    Returns float32 (n, 3) points in the sensor frame (ray order kept)."""
    rng = np.random.default_rng(seed)
    T = pose_matrix(pose)
    o = np.broadcast_to(T[:3, 3], dirs.shape).copy()
    dw = dirs @ T[:3, :3].T
    rng_ = scene.raycast(o, dw, max_range=max_range)
    hit = np.isfinite(rng_)
    if dropout > 0:
        hit &= rng.random(len(dirs)) >= dropout
    r = rng_ + rng.normal(0.0, noise, len(dirs))
    pts = dirs[hit] * r[hit, None]
    if n_keep is not None and len(pts) > n_keep:
        keep = np.sort(rng.choice(len(pts), n_keep, replace=False))
        pts = pts[keep]
    return pts.astype(np.float32)


def odometry(gt_prev, gt_next, cov_diag, seed: int):
    """Noisy relative motion gt_prev^-1 gt_next composed with a tangent
    perturbation drawn from N(0, diag(cov_diag)) (rotation vector, offset).
    Returns (4x4 float64 matrix, 6x6 covariance)."""
    rng = np.random.default_rng(seed)
    D = np.linalg.inv(pose_matrix(gt_prev)) @ pose_matrix(gt_next)
    cov = np.diag(np.asarray(cov_diag, np.float64))
    n = rng.normal(0.0, np.sqrt(np.asarray(cov_diag, np.float64)))
    N = np.eye(4)
    N[:3, :3] = Rotation.from_rotvec(n[:3]).as_matrix()
    N[:3, 3] = n[3:]
    return D @ N, cov


# ---------------------------------------------------------------------------
# complete workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    scene: object
    map_points: np.ndarray
    particles: np.ndarray
    scans: list            # per step: (n, 3) float32 (may be empty)
    odom: list             # per step: 4x4 float64
    odom_cov: list         # per step: 6x6 float64
    gt: np.ndarray         # (n_steps, 7)


def box_room_workload(n_particles: int = 4096, n_steps: int = 10, n_rays: int = 512, scene_seed=1, scan_seed=2,
                      particle_seed=3) -> Workload:
    """Static-scan box room: the same scan, identity odometry, zero noise."""
    room = box_room(scene_seed)
    gt = box_room_gt_pose(room, scan_seed)
    sc = scan(room, gt, spherical_dirs(n_rays), 0.02, scan_seed)
    parts = box_room_particles(n_particles, particle_seed, room.half)
    return Workload("box_room", room, room.map_points, parts, [sc] * n_steps, [np.eye(4)] * n_steps,
                    [np.zeros((6, 6))] * n_steps, np.repeat(gt[None], n_steps, 0))


def outdoor_workload(n_particles: int = 1 << 20, n_steps: int = 100, kidnap_at: int = 50, n_map: int = 1_000_000,
                     n_points: int = 8192, scene_seed=11, traj_seed=12, particle_seed=13, first_step=0,
                     blackout: int = 3) -> Workload:
    gt = outdoor_trajectory(n_steps, kidnap_at, seed=traj_seed)
    scene = outdoor(scene_seed, n_map=n_map, clear_path=gt[:, 4:7])
    gt = outdoor_trajectory(n_steps, kidnap_at, seed=traj_seed, scene=scene)
    parts = outdoor_particles(scene, n_particles, particle_seed)
    dirs = lidar_dirs(32, 512)
    cov_d = np.array([0.01 ** 2] * 3 + [0.05 ** 2] * 3)
    scans, odom, covs = [], [], []
    for s in range(first_step, n_steps):
        if kidnap_at <= s < kidnap_at + blackout:
            scans.append(np.zeros((0, 3), np.float32))
        else:
            scans.append(scan(scene, gt[s], dirs, 0.03, 1000 + s, dropout=0.1, max_range=100.0, n_keep=n_points))
        if s == 0:
            odom.append(np.eye(4)); covs.append(np.diag(cov_d))
        elif s == kidnap_at:
            odom.append(np.eye(4)); covs.append(np.diag(cov_d * 100.0))
        else:
            T, cv = odometry(gt[s - 1], gt[s], cov_d, 2000 + s)
            odom.append(T); covs.append(cv)
    return Workload("outdoor", scene, scene.map_points, parts, scans, odom, covs, gt)
