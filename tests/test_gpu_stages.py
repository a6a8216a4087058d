"""Stage-by-stage parity of the CUDA path (through the C ABI) with the FP64
oracle on the 10 x 10 x 3 m box room (4096 particles, 512-ray scan, 20k map
points, K = C = 16). Tolerances:
  * integers (validity flags, NNF indices, voxel-decided inlier counts, LSH
    keys, bucket order, neighbour sets): bit-exact, except the items the oracle
    flags as ambiguous (an inlier cost within 1e-4 of c_max, a zeta within 1e-9
    of an integer, a K-th/(K+1)-th distance tie within 3e-5);
  * FP32 sums (H, b, log-likelihood): |gpu - ref| <= 1e-4 * sum_k |term_k|;
  * FP64 stages (posterior): 1e-10 relative;
  * SE(3) updates: 1e-5 in angle (rad) and translation (m) per unit of motion.
"""
import numpy as np
import pytest

from gpu_util import check_sums, pose_error, visit_order
from paper_2404_16370_gb300 import synth

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def env(oracle):
    from paper_2404_16370_gb300 import mp
    w = synth.box_room_workload(n_particles=N)
    P = oracle.Params.box_room(N)
    om = oracle.OracleMap(w.map_points, P)
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, N)
    ctx = mp.mp_init_map(w.map_points, params)
    mp.mp_init_particles(ctx, N, poses=w.particles)
    sn, sv, _, covs = oracle.point_normals(w.scans[0], P.r_cov, P.cov_k, P.cov_min, want_covs=True)
    yield dict(mp=mp, w=w, P=P, om=om, ctx=ctx, sn=sn, sv=sv)
    mp.mp_destroy(ctx)


def reset(e, poses=None):
    mp = e["mp"]
    mp.mp_init_particles(e["ctx"], N, poses=e["w"].particles if poses is None else poses)


def normals_agree(gpu_n, ref_n, covs_ref, valid):
    """Normals equal up to sign where the smallest eigenvalue is separated."""
    w = np.linalg.eigvalsh(covs_ref.reshape(-1, 3, 3))
    sep = (w[:, 1] - w[:, 0]) > 1e-3 * np.maximum(w[:, 2], 1e-30)
    m = valid.astype(bool) & sep
    dots = np.abs(np.sum(gpu_n[m].astype(np.float64) * ref_n[m], axis=1))
    return m.sum(), dots.min() if m.any() else 1.0


def test_map_gaussians(env, oracle):
    mp, ctx, om = env["mp"], env["ctx"], env["om"]
    gv = mp.mp_get_buffer(ctx, mp.MP_BUF_MAP_VALID)
    gn = mp.mp_get_buffer(ctx, mp.MP_BUF_MAP_NORMALS)
    assert np.array_equal(gv, om.valid)
    _, _, _, covs = oracle.point_normals(env["w"].map_points, env["P"].r_cov, env["P"].cov_k, env["P"].cov_min,
                                         want_covs=True)
    cnt, worst = normals_agree(gn, om.normals, covs, om.valid)
    assert cnt > 0.9 * len(gv) and worst > 1 - 1e-6


def test_nnf_every_voxel(env):
    mp, ctx, om = env["mp"], env["ctx"], env["om"]
    info = mp.mp_map_info(ctx)
    o, d, inv, off = om.geometry()
    assert np.array_equal(info["origin"], o) and np.array_equal(info["dims"], d)
    assert info["inv_res"] == inv and np.array_equal(info["off"], off)
    vox = np.stack(np.meshgrid(*[np.arange(-2, n + 2) for n in d], indexing="ij"), -1).reshape(-1, 3)
    g = mp.mp_nnf_query(ctx, vox)
    r = om.nnf(vox)
    assert np.array_equal(g, r), f"{(g != r).sum()} of {len(g)} voxels differ"
    assert (r >= 0).sum() > 0.1 * len(r)


def test_scan_gaussians(env, oracle):
    mp, ctx = env["mp"], env["ctx"]
    sc = env["w"].scans[0]
    mp.mp_set_scan(ctx, sc)
    mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN)
    gv = mp.mp_get_buffer(ctx, mp.MP_BUF_SCAN_VALID)
    gn = mp.mp_get_buffer(ctx, mp.MP_BUF_SCAN_NORMALS)
    _, sv, _, covs = oracle.point_normals(sc, env["P"].r_cov, env["P"].cov_k, env["P"].cov_min, want_covs=True)
    assert np.array_equal(gv, sv)
    cnt, worst = normals_agree(gn, env["sn"], covs, sv)
    assert cnt > 0.9 * sv.sum() and worst > 1 - 1e-6


def likelihood_case(env, oracle, poses, scan):
    mp, ctx = env["mp"], env["ctx"]
    reset(env, poses)
    mp.mp_set_scan(ctx, scan)
    mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN | mp.MP_STAGE_LIKELIHOOD)
    gn = mp.mp_get_buffer(ctx, mp.MP_BUF_GN)
    P = env["P"]
    sn, sv, _, _ = oracle.point_normals(scan, P.r_cov, P.cov_k, P.cov_min)
    ref = oracle.likelihood(env["om"], poses, scan, sn, sv, P, amb_tol=1e-4)
    return gn, ref


def check_gn(gn, ref):
    # every particle; exact inlier counts where no decision is ambiguous
    ok = ref["amb"] == 0
    assert ok.mean() > 0.9
    assert np.array_equal(gn[ok, 28].astype(np.int64), ref["n_in"][ok])
    msg = check_sums(gn, ref)
    assert not msg, msg


def test_likelihood_uniform_particles(env, oracle):
    gn, ref = likelihood_case(env, oracle, env["w"].particles, env["w"].scans[0])
    assert (ref["n_in"] > 0).mean() > 0.5
    check_gn(gn, ref)


def test_likelihood_near_ground_truth(env, oracle):
    # particles scattered around the true pose: most points are inliers
    rng = np.random.default_rng(21)
    gt = env["w"].gt[0]
    from scipy.spatial.transform import Rotation
    rot = Rotation.from_quat(gt[:4].astype(np.float64)) * Rotation.from_rotvec(rng.normal(size=(N, 3)) * 0.05)
    poses = np.concatenate([rot.as_quat(), gt[4:] + rng.normal(size=(N, 3)) * 0.1], 1).astype(np.float32)
    gn, ref = likelihood_case(env, oracle, poses, env["w"].scans[0])
    assert np.median(ref["n_in"]) > 0.5 * env["sv"].sum()
    check_gn(gn, ref)


def test_likelihood_sums_do_not_depend_on_the_visiting_order(env):
    """Each particle's sums come from one thread in scan order, so any
    visiting order gives the same bits per particle: identity, reversed,
    a random permutation and the sort stage's position order; the solve reads
    the sums through the same order, so psi agrees too."""
    mp, ctx = env["mp"], env["ctx"]
    reset(env)
    mp.mp_set_scan(ctx, env["w"].scans[0])
    mp.mp_set_step_index(ctx, 2)
    mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN | mp.MP_STAGE_LSH | mp.MP_STAGE_SORT)
    orders = {"position": mp.mp_get_buffer(ctx, mp.MP_BUF_VISIT_ORDER).copy(),
              "identity": np.arange(N, dtype=np.int32), "reversed": np.arange(N, dtype=np.int32)[::-1].copy(),
              "random": np.random.default_rng(5).permutation(N).astype(np.int32)}
    res = {}
    for name, order in orders.items():
        mp.mp_set_buffer(ctx, mp.MP_BUF_VISIT_ORDER, order)
        mp.mp_run_stages(ctx, mp.MP_STAGE_LIKELIHOOD | mp.MP_STAGE_SOLVE)
        res[name] = (mp.mp_get_buffer(ctx, mp.MP_BUF_GN), mp.mp_get_buffer(ctx, mp.MP_BUF_PSI))
    ref_gn, ref_psi = res["position"]
    for name, (gn, psi) in res.items():
        assert np.array_equal(gn.view(np.uint32), ref_gn.view(np.uint32)), name
        assert np.array_equal(psi.view(np.uint32), ref_psi.view(np.uint32)), name


def test_gn_step_solves_the_reference_system(env, oracle):
    mp, ctx = env["mp"], env["ctx"]
    gn, ref = likelihood_case(env, oracle, env["w"].particles, env["w"].scans[0])
    mp.mp_run_stages(ctx, mp.MP_STAGE_SOLVE)
    psi = mp.mp_get_buffer(ctx, mp.MP_BUF_PSI).astype(np.float64)
    P = env["P"]
    Hf = oracle.h_full(ref["H"])
    A = Hf + P.lam * (np.eye(6) * np.diagonal(Hf, axis1=1, axis2=2)[:, :, None]) + P.eps_damp * np.eye(6)
    ok = (ref["amb"] == 0) & (ref["n_in"] >= 6)
    # backward error: psi_gpu solves the reference damped system to 1e-4 relative
    res = np.einsum("nij,nj->ni", A, psi) + ref["b"]
    scale = np.linalg.norm(A, axis=(1, 2)) * np.linalg.norm(psi, axis=1) + np.linalg.norm(ref["b"], axis=1)
    r = np.linalg.norm(res, axis=1) / np.maximum(scale, 1e-30)
    assert r[ok].max() < 1e-4, r[ok].max()
    # forward error where the scaled system is well conditioned
    psi_ref, okr = oracle.gn_solve(ref["H"], ref["b"], ref["n_in"], P)
    d = np.sqrt(np.diagonal(A, axis1=1, axis2=2))
    As = A / d[:, :, None] / d[:, None, :]
    cond = np.linalg.cond(As)
    good = ok & (cond < 1e3)
    rel = np.linalg.norm(psi - psi_ref, axis=1) / np.maximum(np.linalg.norm(psi_ref, axis=1), 1e-12)
    assert good.sum() > 100 and np.percentile(rel[good], 99) < 1e-3
    assert np.all(psi[ref["n_in"] < 6] == 0)


def test_lsh_keys_and_draw(env, oracle):
    mp, ctx, om = env["mp"], env["ctx"], env["om"]
    reset(env)
    mp.mp_set_step_index(ctx, 3)
    mp.mp_run_stages(ctx, mp.MP_STAGE_LSH)
    keys = mp.mp_get_buffer(ctx, mp.MP_BUF_KEYS)
    lsh = mp.mp_get_buffer(ctx, mp.MP_BUF_LSH)
    v = om.valid.astype(bool)
    lo, hi = om.pts[v].min(0).astype(np.float64), om.pts[v].max(0).astype(np.float64)
    q, t, d = oracle.lsh_draw(env["P"].seed, 3, lo, hi, env["P"].lsh_sigma)
    assert np.allclose(lsh, np.concatenate([q, t, d]), rtol=0, atol=1e-14)
    ref = oracle.lsh_keys(env["w"].particles, q, t, d, env["P"])
    ok = ref["flags"] == 0
    assert ok.mean() > 0.999
    assert np.array_equal(keys[ok], ref["keys"][ok])
    assert np.array_equal(mp.mp_get_buffer(ctx, mp.MP_BUF_BUCKETS)[ok], ref["buckets"][ok])


@pytest.mark.parametrize("alpha_scale", [1.0, 0.02])
def test_sort_and_segments(env, oracle, alpha_scale):
    mp = env["mp"]
    P = env["P"]
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, N, alpha=alpha_scale)
    ctx = mp.mp_init_map(env["w"].map_points, params)
    try:
        mp.mp_init_particles(ctx, N, poses=env["w"].particles)
        mp.mp_set_step_index(ctx, 5)
        mp.mp_run_stages(ctx, mp.MP_STAGE_LSH | mp.MP_STAGE_SORT)
        b = mp.mp_get_buffer(ctx, mp.MP_BUF_BUCKETS)
        sid = mp.mp_get_buffer(ctx, mp.MP_BUF_SORTED_IDS)
        seg = mp.mp_get_buffer(ctx, mp.MP_BUF_SEGMENTS)
        visit = mp.mp_get_buffer(ctx, mp.MP_BUF_VISIT_ORDER)
        info = mp.mp_map_info(ctx)
    finally:
        mp.mp_destroy(ctx)
    # the likelihood's visiting order: position cells, LSH order within a cell
    assert np.array_equal(visit, visit_order(sid, env["w"].particles[:, 4:7], info))
    om = env["om"]
    v = om.valid.astype(bool)
    q, t, d = oracle.lsh_draw(P.seed, 5, om.pts[v].min(0).astype(np.float64), om.pts[v].max(0).astype(np.float64),
                              P.lsh_sigma)
    Pa = oracle.Params(**{**P.__dict__, "alpha": alpha_scale})
    ref = oracle.lsh_keys(env["w"].particles, q, t, d, Pa)
    assert ref["flags"].sum() == 0
    assert np.array_equal(b, ref["buckets"])
    s = oracle.bucket_sort(ref["buckets"])
    assert np.array_equal(sid, s["sorted_ids"])
    assert np.array_equal(seg[:, 0], s["seg_lo"]) and np.array_equal(seg[:, 1], s["seg_hi"])
    if alpha_scale < 1:
        assert (s["seg_hi"] - s["seg_lo"]).max() > 16        # crowded buckets exercise the window


def test_neighbour_merge(env, oracle):
    mp, ctx = env["mp"], env["ctx"]
    P = env["P"]
    rng = np.random.default_rng(8)
    old = rng.integers(0, N, (N, P.K)).astype(np.int32)
    old[rng.random((N, P.K)) < 0.3] = -1
    old[:, 0] = np.arange(N)
    reset(env)
    mp.mp_set_buffer(ctx, mp.MP_BUF_NBR_IDS, old)
    mp.mp_set_step_index(ctx, 2)
    mp.mp_run_stages(ctx, mp.MP_STAGE_LSH | mp.MP_STAGE_SORT | mp.MP_STAGE_MERGE)
    ids = mp.mp_get_buffer(ctx, mp.MP_BUF_NBR_IDS)
    kk = mp.mp_get_buffer(ctx, mp.MP_BUF_NBR_K)
    dd = mp.mp_get_buffer(ctx, mp.MP_BUF_NBR_D)
    om = env["om"]
    v = om.valid.astype(bool)
    q, t, d = oracle.lsh_draw(P.seed, 2, om.pts[v].min(0).astype(np.float64), om.pts[v].max(0).astype(np.float64),
                              P.lsh_sigma)
    keys = oracle.lsh_keys(env["w"].particles, q, t, d, P)
    assert keys["flags"].sum() == 0
    srt = oracle.bucket_sort(keys["buckets"])
    ref = oracle.neighbor_merge(env["w"].particles, old, srt, P)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99
    assert np.all(ids[:, 0] == np.arange(N)) and np.all(kk[:, 0] == 1)
    bad = 0
    for i in np.nonzero(ok)[0]:
        gi, ri = ids[i], ref["ids"][i]
        if set(gi[gi >= 0]) != set(ri[ri >= 0]):
            bad += 1
            continue
        # per-neighbour values, matched by id
        order = {j: s for s, j in enumerate(ri)}
        for s_g, j in enumerate(gi):
            if j < 0:
                continue
            s_r = order[j]
            assert abs(kk[i, s_g] - ref["k"][i, s_r]) <= 1e-5 * ref["k"][i, s_r] + 1e-7
            assert np.all(np.abs(dd[i, s_g] - ref["d"][i, s_r]) <= 1e-4 * np.abs(ref["d"][i, s_r]) + 2e-6)
        # stored by decreasing kernel value
        kg = kk[i][gi >= 0]
        assert np.all(np.diff(kg[1:]) <= 1e-6)
    assert bad == 0, f"{bad} neighbour sets differ"


def test_svgd_update(env, oracle):
    mp, ctx = env["mp"], env["ctx"]
    P = env["P"]
    rng = np.random.default_rng(9)
    K = P.K
    ids = rng.integers(0, N, (N, K)).astype(np.int32)
    ids[rng.random((N, K)) < 0.25] = -1
    ids[:, 0] = np.arange(N)
    kk = rng.uniform(0.05, 1.0, (N, K)).astype(np.float32)
    kk[:, 0] = 1
    kk[ids < 0] = 0
    dd = (rng.normal(size=(N, K, 6)) * 0.1).astype(np.float32)
    dd[:, 0] = 0
    psi = (rng.normal(size=(N, 6)) * 0.05).astype(np.float32)
    reset(env)
    for which, arr in ((mp.MP_BUF_NBR_IDS, ids), (mp.MP_BUF_NBR_K, kk), (mp.MP_BUF_NBR_D, dd), (mp.MP_BUF_PSI, psi)):
        mp.mp_set_buffer(ctx, which, arr)
    mp.mp_run_stages(ctx, mp.MP_STAGE_SVGD)
    phi = mp.mp_get_buffer(ctx, mp.MP_BUF_PHI)
    new = mp.mp_get_buffer(ctx, mp.MP_BUF_POSES)
    phi_ref, new_ref = oracle.svgd(env["w"].particles, ids, kk.astype(np.float64), dd.astype(np.float64),
                                   psi.astype(np.float64), P)
    assert np.allclose(phi, phi_ref, rtol=1e-5, atol=1e-6)
    ang, dist = pose_error(new, new_ref)
    mag = 1 + np.linalg.norm(phi_ref, axis=1)
    assert np.all(ang <= 1e-5 * mag) and np.all(dist <= 2e-6 * (1 + np.abs(new_ref[:, 4:]).max(1)) * mag)


def test_svgd_update_preconditioned(env, oracle):
    """svgd_precond = 1: k_solve's damped inverse and k_svgd's product against
    the oracle's Eq. 6 with the repulsion times numpy's inverse, on the same
    lists, steps and Gauss-Newton sums (from a full pass of the stages)."""
    mp = env["mp"]
    P = env["P"]
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, N)
    params.svgd_precond = 1
    ctx = mp.mp_init_map(env["w"].map_points, params)
    try:
        mp.mp_init_particles(ctx, N, poses=env["w"].particles)
        mp.mp_set_scan(ctx, env["w"].scans[0])
        mp.mp_run_stages(ctx, mp.MP_STAGE_SCAN | mp.MP_STAGE_LSH | mp.MP_STAGE_SORT | mp.MP_STAGE_MERGE)
        mp.mp_run_stages(ctx, mp.MP_STAGE_LIKELIHOOD | mp.MP_STAGE_SOLVE)
        g = {k: mp.mp_get_buffer(ctx, b) for k, b in (("ids", mp.MP_BUF_NBR_IDS), ("k", mp.MP_BUF_NBR_K),
                                                     ("d", mp.MP_BUF_NBR_D), ("psi", mp.MP_BUF_PSI),
                                                     ("gn", mp.MP_BUF_GN), ("poses", mp.MP_BUF_POSES))}
        mp.mp_run_stages(ctx, mp.MP_STAGE_SVGD)
        phi = mp.mp_get_buffer(ctx, mp.MP_BUF_PHI)
    finally:
        mp.mp_destroy(ctx)
    H = g["gn"][:, :21].astype(np.float64)      # exported in particle order
    ok = (g["gn"][:, 28] >= 6) & np.any(g["psi"] != 0, axis=1)
    pinv = oracle.svgd_precond_matrices(H, ok, P)
    phi_ref, _ = oracle.svgd(g["poses"], g["ids"], g["k"].astype(np.float64), g["d"].astype(np.float64),
                             g["psi"].astype(np.float64), P, pinv)
    assert ok.mean() > 0.3
    scale = 1e-6 + np.abs(phi_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(phi - phi_ref) <= 2e-4 * scale)
    # the preconditioned repulsion is far weaker than the printed one
    phi_lit, _ = oracle.svgd(g["poses"], g["ids"], g["k"].astype(np.float64), g["d"].astype(np.float64),
                             g["psi"].astype(np.float64), P)
    assert np.median(np.linalg.norm(phi_ref, axis=1)) < np.median(np.linalg.norm(phi_lit, axis=1))


def test_posterior(env, oracle):
    mp, ctx = env["mp"], env["ctx"]
    P = env["P"]
    rng = np.random.default_rng(10)
    K = P.K
    ids = rng.integers(0, N, (N, K)).astype(np.int32)
    ids[rng.random((N, K)) < 0.25] = -1
    ids[:, 0] = np.arange(N)
    kk = rng.uniform(0.05, 1.0, (N, K)).astype(np.float32)
    kk[:, 0] = 1
    loglik = (-rng.uniform(0, 60, N)).astype(np.float32)
    logprior = -rng.uniform(0, 5, N)
    logprior[::97] = -np.inf                        # zero prior mass survives only through Eq. 11
    reset(env)
    mp.mp_set_buffer(ctx, mp.MP_BUF_NBR_IDS, ids)
    mp.mp_set_buffer(ctx, mp.MP_BUF_NBR_K, kk)
    mp.mp_set_buffer(ctx, mp.MP_BUF_LOGLIK, loglik)
    mp.mp_set_buffer(ctx, mp.MP_BUF_LOG_PRIOR, logprior)
    mp.mp_run_stages(ctx, mp.MP_STAGE_POSTERIOR)
    post = mp.mp_get_buffer(ctx, mp.MP_BUF_POST)
    p0 = mp.mp_get_buffer(ctx, mp.MP_BUF_POST_INIT)
    lp = mp.mp_get_buffer(ctx, mp.MP_BUF_LOG_PRIOR)
    best, best_p = mp.mp_get_posterior(ctx)
    p0_ref, p_ref, b_ref = oracle.posterior(logprior, loglik.astype(np.float64), ids, kk.astype(np.float64),
                                            P.post_iters, P.post_floor)
    assert np.allclose(p0, p0_ref, rtol=1e-10, atol=1e-300)
    assert np.allclose(post, p_ref, rtol=1e-10, atol=1e-300)
    assert abs(post.sum() - 1) < 1e-12
    with np.errstate(divide="ignore"):
        assert np.allclose(lp, np.log(p_ref), rtol=1e-10)
    assert np.array_equal(best, env["w"].particles[b_ref]) and abs(best_p - p_ref[b_ref]) < 1e-12


def test_prediction(env, oracle):
    mp, ctx = env["mp"], env["ctx"]
    reset(env)
    from scipy.spatial.transform import Rotation
    T = np.eye(4)
    T[:3, :3] = Rotation.from_rotvec([0.02, -0.03, 0.2]).as_matrix()
    T[:3, 3] = [0.7, -0.2, 0.05]
    cov = np.diag([1e-4] * 3 + [2.5e-3] * 3)
    cov[3, 4] = cov[4, 3] = 1e-3
    mp.mp_set_odometry(ctx, T, cov)
    mp.mp_set_step_index(ctx, 7)
    mp.mp_run_stages(ctx, mp.MP_STAGE_PREDICT)
    got = mp.mp_get_buffer(ctx, mp.MP_BUF_POSES)
    ref, _ = oracle.predict(env["w"].particles, T, cov, env["P"].seed, 7)
    ang, dist = pose_error(got, ref)
    assert ang.max() < 2e-6 and dist.max() < 5e-6


def test_full_step_matches_oracle(env, oracle):
    """One complete mp_step from the uniform start against OracleFilter.step:
    LSH keys bit for bit; neighbour sets; log-likelihoods; the SVGD update phi
    and the updated poses of every particle whose own and neighbours' sums are
    unambiguous and whose neighbours' Gauss-Newton systems are well
    conditioned (cond < 1e6), to 1e-4 max(1, |phi|); the posterior element by
    element: against the oracle's posterior of the GPU's own log-likelihoods
    and lists to 1e-10, and against the oracle's own step within the bound
    its log-likelihood and kernel-weight differences allow; the
    representative state."""
    mp = env["mp"]
    P = env["P"]
    params = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, N)
    ctx = mp.mp_init_map(env["w"].map_points, params)
    try:
        mp.mp_init_particles(ctx, N, poses=env["w"].particles)
        sc = env["w"].scans[0]
        mp.mp_step(ctx, sc, np.eye(4), np.zeros((6, 6)))
        best, best_p = mp.mp_get_posterior(ctx)
        g = {k: mp.mp_get_buffer(ctx, b) for k, b in (("ids", mp.MP_BUF_NBR_IDS), ("gn", mp.MP_BUF_GN),
                                                     ("poses", mp.MP_BUF_POSES), ("post", mp.MP_BUF_POST),
                                                     ("keys", mp.MP_BUF_KEYS), ("phi", mp.MP_BUF_PHI),
                                                     ("k", mp.MP_BUF_NBR_K), ("loglik", mp.MP_BUF_LOGLIK))}
    finally:
        mp.mp_destroy(ctx)
    f = oracle.OracleFilter(env["om"], P, env["w"].particles.copy())
    out = f.step(sc)
    assert out["lsh_flags"].sum() == 0 and np.array_equal(g["keys"], out["keys"])
    ok = (out["merge_flags"] == 0) & (out["amb"] == 0)
    same = np.array([set(a[a >= 0]) == set(b[b >= 0]) for a, b in zip(g["ids"], out["nbr_ids"])])
    assert same[ok].all()
    err_ll = np.abs(g["gn"][:, 27] - out["loglik"])
    assert np.all(err_ll[ok] <= 1e-4 * np.abs(out["loglik"][ok]) + 1e-3)
    # SVGD update and poses: particles whose neighbourhood is unambiguous and well conditioned
    H = oracle.h_full(out["H"])
    well = np.linalg.cond(H + P.lam * np.einsum("nii->ni", H)[:, :, None] * np.eye(6) + P.eps_damp * np.eye(6)) < 1e6
    good = ok & well
    ids = out["nbr_ids"]
    hood = np.array([good[i] and bool(np.all(good[row[row >= 0]])) for i, row in enumerate(ids)])
    assert hood.sum() > N // 4, hood.sum()
    scale = np.maximum(1.0, np.linalg.norm(out["phi"], axis=1))
    assert np.all(np.abs(g["phi"] - out["phi"]).max(axis=1)[hood] <= 1e-4 * scale[hood])
    ang, dist = pose_error(g["poses"], out["new_poses"])
    assert np.all(ang[hood] <= 1e-4 * scale[hood]) and np.all(dist[hood] <= 1e-4 * scale[hood])
    # the posterior: the GPU's step on its own log-likelihoods and lists, element by element
    _, p_own, b_own = oracle.posterior(None, g["loglik"].astype(np.float64), g["ids"], g["k"].astype(np.float64),
                                       P.post_iters, P.post_floor)
    assert np.allclose(g["post"], p_own, rtol=1e-10, atol=1e-300)
    # and against the oracle's own step (lists equal): with every log-likelihood within dl of
    # the oracle's, each posterior moves by at most a factor exp(4 dl) (Eq. 11 is a positive
    # linear map); the FP32 kernel weights add 1e-6 relative and, where a weight underflows
    # FP32 (k < 1e-38), an absolute 1e-36 of the total mass
    if same.all():
        d = 4 * err_ll.max() + 1e-9
        tol = (np.expm1(d) + 1e-6) * out["post"] + 1e-36
        assert np.all(np.abs(g["post"] - out["post"]) <= tol), np.max(np.abs(g["post"] - out["post"]) - tol)
    # the representative state: same particle unless its log-posterior ties within the tolerance
    lp_ref = np.log(np.maximum(out["post"], 1e-300))
    top2 = np.sort(lp_ref)[-2:]
    if top2[1] - top2[0] > 1e-2:
        assert np.array_equal(best, out["best_pose"]) or pose_error(best[None], out["best_pose"][None])[0][0] < 1e-4
    assert abs(g["post"].sum() - 1) < 1e-12
