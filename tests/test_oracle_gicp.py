"""Pins of the oracle's scan-to-scan GICP odometry (Sec. III-B): exact
recovery of a rigid motion between a scan and its own transformed copy, the
true motion between two ray-cast scans, and the degenerate directions of a
planar scene showing up in Sigma^DeltaT = H^-1."""
import numpy as np
from scipy.spatial.transform import Rotation

from paper_2404_16370_gb300 import synth


def _T(rotvec, t):
    T = np.eye(4)
    T[:3, :3] = Rotation.from_rotvec(rotvec).as_matrix()
    T[:3, 3] = t
    return T


def _err(Ta, Tb):
    D = np.linalg.inv(Ta) @ Tb
    return Rotation.from_matrix(D[:3, :3]).magnitude(), np.linalg.norm(D[:3, 3])


def test_recovers_a_rigid_motion_exactly(oracle):
    P = oracle.Params.box_room()
    room = synth.box_room(1)
    gt = synth.box_room_gt_pose(room, 2)
    tgt = synth.scan(room, gt, synth.spherical_dirs(512), 0.0, 2)
    T_true = _T([0.01, -0.02, 0.03], [0.08, -0.05, 0.02])
    # the same points seen from the moved sensor: src = T_true^-1 tgt
    src = ((tgt.astype(np.float64) - T_true[:3, 3]) @ T_true[:3, :3]).astype(np.float32)
    out = oracle.gicp(src, tgt, P, max_iters=50, tol=1e-12)
    ang, dist = _err(out["T"], T_true)
    assert ang < 1e-7 and dist < 1e-6
    # every source point with a Gaussian finds its own copy
    _, sv, _, _ = oracle.point_normals(src, P.r_cov, P.cov_k, P.cov_min)
    _, tv, _, _ = oracle.point_normals(tgt, P.r_cov, P.cov_k, P.cov_min)
    assert out["n_corr"] >= int(np.sum(sv.astype(bool) & tv.astype(bool)))


def test_matches_the_true_motion_between_scans(oracle):
    P = oracle.Params.box_room()
    room = synth.box_room(1)
    p0 = synth.box_room_gt_pose(room, 3)
    T0 = synth.pose_matrix(p0)
    T1 = T0 @ _T([0.0, 0.0, 0.05], [0.15, 0.05, 0.0])
    dirs = synth.spherical_dirs(2048)
    s0 = synth.scan(room, p0, dirs, 0.0, 1)
    s1 = synth.scan(room, synth.matrix_pose(T1), dirs, 0.0, 1)
    out = oracle.gicp(s1, s0, P)
    ang, dist = _err(out["T"], np.linalg.inv(T0) @ T1)
    assert ang < np.deg2rad(0.3) and dist < 0.02
    assert np.all(np.linalg.eigvalsh(out["cov"]) > 0)


def test_planar_scene_is_degenerate_in_plane(oracle):
    """Points on the plane z = 0 only: in-plane translation and yaw leave the
    cost unchanged, so H is (near) singular there and Sigma^DeltaT is large
    in those directions compared with the constrained ones."""
    P = oracle.Params.box_room()
    rng = np.random.default_rng(0)
    xy = rng.uniform(-3, 3, (1500, 2))
    tgt = np.concatenate([xy, np.zeros((1500, 1))], 1).astype(np.float32)
    src = tgt.copy()
    out = oracle.gicp(src, tgt, P, max_iters=3)
    Hm = np.zeros((6, 6))
    Hm[np.triu_indices(6)] = out["H"]
    Hm = Hm + np.triu(Hm, 1).T
    w, V = np.linalg.eigh(Hm)
    # three directions (rot z, t x, t y) carry only the in-plane weight eps
    free = np.abs(V[:, :3])
    assert w[2] < 1e-2 * w[3]
    assert np.all(free[[2, 3, 4], :].sum(0) > 0.99)
