"""Scan-to-scan GICP odometry on the GPU (mp_gicp, mp_step_gicp) against the
FP64 oracle (oracle.gicp): the same motion estimate and Hessian on ray-cast
box-room scan pairs, exact recovery of a rigid motion, and a filter that
tracks the sensor with GICP odometry instead of given odometry."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2404_16370_gb300 import synth

pytestmark = pytest.mark.gpu


def _T(rotvec, t):
    T = np.eye(4)
    T[:3, :3] = Rotation.from_rotvec(rotvec).as_matrix()
    T[:3, 3] = t
    return T


def _err(Ta, Tb):
    D = np.linalg.inv(Ta) @ Tb
    return Rotation.from_matrix(D[:3, :3]).magnitude(), np.linalg.norm(D[:3, 3])


@pytest.fixture(scope="module")
def ctx():
    from paper_2404_16370_gb300 import mp
    room = synth.box_room(1)
    c = mp.mp_init_map(room.map_points, mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 1024))
    mp.mp_init_particles(c, 1024, poses=synth.box_room_particles(1024, 3, room.half))
    yield room, c
    mp.mp_destroy(c)


@pytest.mark.parametrize("motion", [([0.0, 0.0, 0.05], [0.15, 0.05, 0.0]), ([0.02, -0.01, -0.08], [-0.1, 0.2, 0.05])])
def test_gicp_matches_oracle(ctx, oracle, motion):
    from paper_2404_16370_gb300 import mp
    room, c = ctx
    P = oracle.Params.box_room()
    p0 = synth.box_room_gt_pose(room, 3)
    T0 = synth.pose_matrix(p0)
    T1 = T0 @ _T(*motion)
    dirs = synth.spherical_dirs(2048)
    s0 = synth.scan(room, p0, dirs, 0.02, 1)
    s1 = synth.scan(room, synth.matrix_pose(T1), dirs, 0.02, 2)
    g = mp.mp_gicp(c, s1, s0)
    r = oracle.gicp(s1, s0, P)
    ang, dist = _err(g["T"], r["T"])
    assert ang < 1e-5 and dist < 1e-5, (ang, dist)
    assert abs(g["n_corr"] - r["n_corr"]) <= 3
    # the Hessian at the result: its inverse within 1e-3 of its scale
    assert np.abs(g["cov"] - r["cov"]).max() <= 1e-3 * np.abs(r["cov"]).max()
    # and the true motion within the scans' noise
    ang_t, dist_t = _err(g["T"], np.linalg.inv(T0) @ T1)
    assert ang_t < np.deg2rad(0.5) and dist_t < 0.03


def test_gicp_recovers_a_rigid_motion(ctx):
    from paper_2404_16370_gb300 import mp
    room, c = ctx
    gt = synth.box_room_gt_pose(room, 2)
    tgt = synth.scan(room, gt, synth.spherical_dirs(1024), 0.0, 2)
    T_true = _T([0.01, -0.02, 0.03], [0.08, -0.05, 0.02])
    src = ((tgt.astype(np.float64) - T_true[:3, 3]) @ T_true[:3, :3]).astype(np.float32)
    g = mp.mp_gicp(c, src, tgt, max_iters=50)
    ang, dist = _err(g["T"], T_true)
    assert ang < 2e-6 and dist < 2e-6


def test_filter_tracks_with_gicp_odometry():
    """Particles around the start pose, the sensor moving 0.1 m and 1 degree
    a step: with odometry from GICP the representative state stays within
    0.1 m / 2 degrees of the truth over 12 steps."""
    from paper_2404_16370_gb300 import mp
    room = synth.box_room(1)
    p = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 4096)
    p.svgd_precond = 1
    c = mp.mp_init_map(room.map_points, p)
    try:
        T = synth.pose_matrix(synth.box_room_gt_pose(room, 5))
        step = _T([0.0, 0.0, np.deg2rad(1.0)], [0.1, 0.0, 0.0])
        parts = synth.tracking_particles(synth.matrix_pose(T), 4096, seed=3, sigma_t=0.05, sigma_r=0.01)
        mp.mp_init_particles(c, 4096, poses=parts)
        dirs = synth.spherical_dirs(1024)
        errs = []
        for s in range(12):
            if s:
                T = T @ step
            sc = synth.scan(room, synth.matrix_pose(T), dirs, 0.02, 100 + s)
            mp.mp_step_gicp(c, sc, cov_scale=1.0)
            best, _ = mp.mp_get_posterior(c)
            errs.append(_err(synth.pose_matrix(best), T))
        errs = np.array(errs)
        print("\nmax error", errs[:, 1].max(), "m", np.rad2deg(errs[:, 0].max()), "deg")
        assert errs[:, 1].max() < 0.1 and errs[:, 0].max() < np.deg2rad(2.0)
    finally:
        mp.mp_destroy(c)
