"""Pins of the oracle's likelihood and Gauss-Newton terms (Sec. III-C, Eq. 2-4):
finite differences of the residual and of the frozen-information cost, the
zero-residual Hessian, a one-step exact recovery of a pure translation offset,
an off-map particle, and the information matrices recomputed with
numpy.linalg.inv."""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

from paper_2404_16370_gb300 import synth


def hat(xi):
    w, v = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def pose_mat(p):
    q = np.asarray(p[:4], np.float64)
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(q).as_matrix()
    T[:3, 3] = p[4:7]
    return T


def patches(spacing=0.25):
    """Four separated planar lattice patches (spacing > sqrt(3) * 0.1 m)."""
    a = np.arange(-1.5, 1.5 + 1e-9, spacing)
    A, B = np.meshgrid(a, a, indexing="ij")
    A, B = A.ravel(), B.ravel()
    floor = np.stack([A, B, np.zeros_like(A)], -1)
    wall_x = np.stack([np.full_like(A, 2.5), A, B + 2.0], -1)
    wall_y = np.stack([A, np.full_like(A, 2.5), B + 2.0], -1)
    n = np.array([1.0, 1.0, 1.0]) / np.sqrt(3)
    u = np.array([1.0, -1.0, 0.0]) / np.sqrt(2)
    v = np.cross(n, u)
    tilt = np.array([-2.5, -2.5, 2.0]) + A[:, None] * u + B[:, None] * v
    return np.concatenate([floor, wall_x, wall_y, tilt]).astype(np.float32)


@pytest.fixture(scope="module")
def stationary(oracle):
    P = oracle.Params(res=0.1, r_max=0.5, r_cov=0.6, c_max=9.0)
    pts = patches()
    m = oracle.OracleMap(pts, P)
    rot = Rotation.from_euler("ZYX", [0.4, -0.15, 0.1])
    t_gt = np.array([0.3, -0.2, 1.0])
    gt = np.concatenate([rot.as_quat(), t_gt]).astype(np.float32)
    T = pose_mat(gt)
    scan = ((pts.astype(np.float64) - T[:3, 3]) @ T[:3, :3]).astype(np.float32)   # R^T (p - t)
    sn, sv, _, _ = oracle.point_normals(scan, P.r_cov, P.cov_k, P.cov_min)
    return dict(P=P, map=m, pts=pts, gt=gt, scan=scan, sn=sn, sv=sv)


def test_stationary_point(oracle, stationary):
    s = stationary
    lk = oracle.likelihood(s["map"], s["gt"][None], s["scan"], s["sn"], s["sv"], s["P"])
    pairs = oracle.likelihood_pairs(s["map"], s["gt"], s["scan"], s["sn"], s["sv"], s["P"])
    assert s["sv"].all()
    assert np.array_equal(pairs["m"], np.arange(len(s["scan"])))     # each point finds itself
    assert lk["n_in"][0] == len(s["scan"])
    H = oracle.h_full(lk["H"])[0]
    assert abs(lk["loglik"][0]) < 1e-6
    assert np.abs(lk["b"][0]).max() < 1e-5 * np.abs(H).max()
    psi, ok = oracle.gn_solve(lk["H"], lk["b"], lk["n_in"], s["P"])
    assert ok[0] == 1 and np.abs(psi).max() < 1e-5


def frozen_cost(xi, pose, pairs, scan, map_pts):
    T = pose_mat(pose) @ expm(hat(xi))
    f = 0.0
    for k in np.nonzero(pairs["inlier"])[0]:
        e = map_pts[pairs["m"][k]].astype(np.float64) - (T[:3, :3] @ scan[k].astype(np.float64) + T[:3, 3])
        f += e @ pairs["omega"][k] @ e
    return f


def test_fd_hessian_at_zero_residual(oracle, stationary):
    s = stationary
    lk = oracle.likelihood(s["map"], s["gt"][None], s["scan"], s["sn"], s["sv"], s["P"])
    pairs = oracle.likelihood_pairs(s["map"], s["gt"], s["scan"], s["sn"], s["sv"], s["P"])
    H = oracle.h_full(lk["H"])[0]
    h = 1e-4
    Hfd = np.zeros((6, 6))
    E = np.eye(6)
    for a in range(6):
        for b in range(a, 6):
            f = lambda x: frozen_cost(x, s["gt"], pairs, s["scan"], s["pts"])
            Hfd[a, b] = (f(h * (E[a] + E[b])) - f(h * (E[a] - E[b])) - f(h * (E[b] - E[a])) + f(-h * (E[a] + E[b]))) / (4 * h * h)
            Hfd[b, a] = Hfd[a, b]
    assert np.allclose(Hfd, 2 * H, rtol=1e-5, atol=1e-5 * np.abs(H).max())


def test_translation_offset_recovered_in_one_step(oracle, stationary):
    s = stationary
    P0 = oracle.Params(**{**s["P"].__dict__, "lam": 0.0, "eps_damp": 0.0})
    dt = np.array([0.012, -0.017, 0.009])
    pose = s["gt"].copy()
    pose[4:] = (s["gt"][4:].astype(np.float64) + dt).astype(np.float32)
    pairs = oracle.likelihood_pairs(s["map"], pose, s["scan"], s["sn"], s["sv"], P0)
    assert np.array_equal(pairs["m"], np.arange(len(s["scan"])))
    lk = oracle.likelihood(s["map"], pose[None], s["scan"], s["sn"], s["sv"], P0)
    psi, ok = oracle.gn_solve(lk["H"], lk["b"], lk["n_in"], P0)
    R = pose_mat(pose)[:3, :3]
    true_dt = pose[4:].astype(np.float64) - s["gt"][4:].astype(np.float64)
    assert np.allclose(psi[0, :3], 0, atol=2e-6)
    assert np.allclose(psi[0, 3:], -R.T @ true_dt, atol=2e-6)


@pytest.fixture(scope="module")
def room_case(oracle):
    w = synth.box_room_workload(n_particles=64)
    P = oracle.Params.box_room(64)
    m = oracle.OracleMap(w.map_points, P)
    sc = w.scans[0]
    sn, sv, _, _ = oracle.point_normals(sc, P.r_cov, P.cov_k, P.cov_min)
    gt = w.gt[0]
    near = gt.copy()
    near[4:] += np.array([0.05, -0.04, 0.03], np.float32)
    near[:4] = (Rotation.from_quat(gt[:4].astype(np.float64)) * Rotation.from_rotvec([0.02, -0.01, 0.03])).as_quat()
    return dict(w=w, P=P, map=m, scan=sc, sn=sn, sv=sv, pose=near.astype(np.float32))


def test_fd_gradient_is_twice_b(oracle, room_case):
    c = room_case
    pairs = oracle.likelihood_pairs(c["map"], c["pose"], c["scan"], c["sn"], c["sv"], c["P"])
    lk = oracle.likelihood(c["map"], c["pose"][None], c["scan"], c["sn"], c["sv"], c["P"])
    assert pairs["inlier"].sum() == lk["n_in"][0] > 50
    h = 1e-6
    g = np.zeros(6)
    for a in range(6):
        e = np.zeros(6)
        e[a] = h
        g[a] = (frozen_cost(e, c["pose"], pairs, c["scan"], c["w"].map_points)
                - frozen_cost(-e, c["pose"], pairs, c["scan"], c["w"].map_points)) / (2 * h)
    b = lk["b"][0]
    assert np.allclose(g, 2 * b, rtol=1e-4, atol=1e-5 * np.abs(b).max())


def test_residual_jacobian_fd(oracle, room_case):
    c = room_case
    pairs = oracle.likelihood_pairs(c["map"], c["pose"], c["scan"], c["sn"], c["sv"], c["P"])
    T = pose_mat(c["pose"])
    h = 1e-6
    for k in np.nonzero(pairs["m"] >= 0)[0][:40]:
        mu_m = c["w"].map_points[pairs["m"][k]].astype(np.float64)
        mu = c["scan"][k].astype(np.float64)
        Jfd = np.zeros((3, 6))
        for a in range(6):
            e = np.zeros(6)
            e[a] = h
            Tp, Tm = T @ expm(hat(e)), T @ expm(hat(-e))
            Jfd[:, a] = ((mu_m - Tp[:3, :3] @ mu - Tp[:3, 3]) - (mu_m - Tm[:3, :3] @ mu - Tm[:3, 3])) / (2 * h)
        assert np.allclose(pairs["J"][k], Jfd, atol=1e-6 * max(1, np.abs(mu).max()))


def test_information_and_cost_by_numpy(oracle, room_case):
    c = room_case
    P = c["P"]
    pairs = oracle.likelihood_pairs(c["map"], c["pose"], c["scan"], c["sn"], c["sv"], P)
    lk = oracle.likelihood(c["map"], c["pose"][None], c["scan"], c["sn"], c["sv"], P)
    R = pose_mat(c["pose"])[:3, :3]
    total = 0.0
    for k in range(len(c["scan"])):
        if not c["sv"][k]:
            assert pairs["m"][k] == -2
            continue
        if pairs["m"][k] < 0:
            total -= P.c_max
            continue
        nm = c["map"].normals[pairs["m"][k]]
        ns = c["sn"][k]
        SM = np.eye(3) - (1 - P.eps_cov) * np.outer(nm, nm)
        SS = np.eye(3) - (1 - P.eps_cov) * np.outer(ns, ns)
        Om = np.linalg.inv(SM + R @ SS @ R.T)
        assert np.allclose(pairs["omega"][k], Om, rtol=1e-6, atol=1e-6 * np.abs(Om).max())
        cst = pairs["e"][k] @ Om @ pairs["e"][k]
        assert np.isclose(pairs["c"][k], cst, rtol=1e-6, atol=1e-9)
        total -= min(cst, P.c_max)
    assert np.isclose(lk["loglik"][0], total, rtol=1e-6)   # R here from the normalised quaternion


def test_off_map_particle(oracle, room_case):
    c = room_case
    far = c["pose"].copy()
    far[4:] = [1000.0, -1000.0, 500.0]
    lk = oracle.likelihood(c["map"], far[None], c["scan"], c["sn"], c["sv"], c["P"])
    assert lk["loglik"][0] == -c["P"].c_max * int(c["sv"].sum())
    assert lk["n_in"][0] == 0 and np.all(lk["H"] == 0) and np.all(lk["b"] == 0)


def test_gn_solve_matches_numpy(oracle):
    rng = np.random.default_rng(9)
    n = 50
    A = rng.normal(size=(n, 6, 6))
    Hf = A @ A.transpose(0, 2, 1) + 0.1 * np.eye(6)
    iu = np.triu_indices(6)
    H21 = Hf[:, iu[0], iu[1]]
    b = rng.normal(size=(n, 6))
    n_in = np.full(n, 100, np.int32)
    n_in[3] = 5
    P = oracle.Params()
    psi, ok = oracle.gn_solve(H21, b, n_in, P)
    for i in range(n):
        if i == 3:
            assert ok[i] == 0 and np.all(psi[i] == 0)
            continue
        M = Hf[i] + P.lam * np.diag(np.diag(Hf[i])) + P.eps_damp * np.eye(6)
        assert np.allclose(psi[i], np.linalg.solve(M, -b[i]), rtol=1e-10, atol=1e-12)


def test_ambiguity_band_bounds_the_other_decision(oracle, room_case):
    """amb / ambabs: an inlier decision within amb_tol * c_max of the
    threshold is ambiguous, and ambabs bounds how far each output moves if
    the other decision is taken. Straddle one pair's cost c_j with two
    thresholds c_j (1 +- d): the pair is an inlier under the first and an
    outlier under the second, no other pair changes side (the band holds only
    it), and the outputs of the two runs differ by exactly that pair's terms,
    which both runs report in ambabs."""
    c = room_case
    pairs = oracle.likelihood_pairs(c["map"], c["pose"], c["scan"], c["sn"], c["sv"], c["P"])
    costs = pairs["c"][pairs["m"] >= 0]
    costs = np.sort(costs)
    gaps = np.diff(costs)
    # a pair whose cost is well separated from its neighbours and in the middle of the range
    cand = [k for k in range(1, len(costs) - 1) if min(gaps[k - 1], gaps[k]) > 1e-3 * costs[k] and 0.5 < costs[k] < 50]
    assert cand, "no isolated pair cost"
    cj = costs[cand[len(cand) // 2]]
    d = 1e-6
    tol = 1e-4   # band half-width (relative to c_max): holds c_j under both thresholds, no other pair
    out = {}
    for side, cm in (("in", cj * (1 + d)), ("out", cj * (1 - d))):
        P = oracle.Params(**{**c["P"].__dict__, "c_max": cm})
        out[side] = oracle.likelihood(c["map"], c["pose"][None], c["scan"], c["sn"], c["sv"], P, amb_tol=tol)
        assert out[side]["amb"][0] == 1
    A, B = out["in"], out["out"]
    assert A["n_in"][0] == B["n_in"][0] + 1
    dH = np.abs(A["H"][0] - B["H"][0])
    db = np.abs(A["b"][0] - B["b"][0])
    for r in (A, B):
        assert np.allclose(r["ambabs"][0, :21], dH, rtol=1e-9, atol=1e-12 * np.abs(A["H"]).max())
        assert np.allclose(r["ambabs"][0, 21:27], db, rtol=1e-9, atol=1e-12 * np.abs(A["b"]).max())
    assert dH.max() > 0 and db.max() > 0
    # log p = -(sum of inlier costs) - c_max (outliers): with N_out outliers
    # under the first threshold the two differ by -d c_j (2 N_out + 1)
    n_out = int(c["sv"].sum()) - int(A["n_in"][0])
    assert np.isclose(A["loglik"][0] - B["loglik"][0], -d * cj * (2 * n_out + 1), rtol=1e-6, atol=1e-9)
    assert np.isclose(A["ambabs"][0, 27], d * cj, rtol=1e-6) and np.isclose(B["ambabs"][0, 27], d * cj, rtol=1e-6)
