"""Pins of the oracle's SVGD update (Eq. 5, 6), posterior propagation (Eq. 11),
prediction (Eq. 1), Philox stream and uniform initialisation: a lone particle
reduces to the Gauss-Newton step, all-pairs SVGD computed with
scipy.linalg.expm/logm, the kernel gradient by finite differences, the
hand-derived 4-ring (tests/golden/posterior_ring4.json), fixed points of
Eq. 11, numpy's Cholesky, and distribution checks of the random streams."""
import json
import os

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import expm, logm
from scipy.spatial.transform import Rotation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def hat(xi):
    w, v = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def vee(M):
    return np.array([M[2, 1], M[0, 2], M[1, 0], M[0, 3], M[1, 3], M[2, 3]])


def mat(p):
    p = np.asarray(p, np.float64)
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(p[:4] / np.linalg.norm(p[:4])).as_matrix()
    T[:3, 3] = p[4:7]
    return T


def test_lone_particle_follows_gn_step(oracle):
    P = oracle.Params()
    pose = np.array([0.1, -0.2, 0.3, 0.9, 1.0, 2.0, -1.0])
    pose[:4] /= np.linalg.norm(pose[:4])
    pose = pose.astype(np.float32)[None]
    ids = np.full((1, 4), -1, np.int32); ids[0, 0] = 0
    kk = np.zeros((1, 4)); kk[0, 0] = 1.0
    dd = np.zeros((1, 4, 6))
    psi = np.array([[0.05, -0.02, 0.01, 0.3, -0.1, 0.2]])
    phi, out = oracle.svgd(pose, ids, kk, dd, psi, P)
    assert np.allclose(phi, psi, atol=1e-15)
    assert np.allclose(mat(out[0]), mat(pose[0]) @ expm(hat(psi[0])), atol=1e-12)


def test_all_pairs_svgd(oracle):
    # K = N: Eq. 6 is SVGD over all particles; kernel values and d_ij from logm.
    rng = np.random.default_rng(1)
    n = 7
    rot = Rotation.from_rotvec(rng.normal(size=(n, 3)) * 0.2)
    poses = np.concatenate([rot.as_quat(), rng.normal(size=(n, 3)) * 0.4], 1).astype(np.float32)
    P = oracle.Params(alpha=0.0, K=n, C=n, nb_log2=3)
    srt = oracle.bucket_sort(np.zeros(n, np.uint32))
    mg = oracle.neighbor_merge(poses, None, srt, P)
    psi = rng.normal(size=(n, 6)) * 0.1
    phi, out = oracle.svgd(poses, mg["ids"], mg["k"], mg["d"], psi, P)
    W = np.array([5.0] * 3 + [2.5] * 3)
    Ts = [mat(p) for p in poses]
    for i in range(n):
        num = np.zeros(6); den = 0.0
        for j in range(n):
            d = vee(np.real(logm(np.linalg.inv(Ts[i]) @ Ts[j]))) if j != i else np.zeros(6)
            k = np.exp(-(W * d * d).sum())
            num += k * psi[j] - 2 * k * W * d
            den += k
        assert np.allclose(phi[i], num / den, atol=1e-9)
        assert np.allclose(mat(out[i]), Ts[i] @ expm(hat(num / den)), atol=1e-9)


def _all_pairs_case(oracle, n=7, seed=1):
    rng = np.random.default_rng(seed)
    rot = Rotation.from_rotvec(rng.normal(size=(n, 3)) * 0.2)
    poses = np.concatenate([rot.as_quat(), rng.normal(size=(n, 3)) * 0.4], 1).astype(np.float32)
    P = oracle.Params(alpha=0.0, K=n, C=n, nb_log2=3)
    srt = oracle.bucket_sort(np.zeros(n, np.uint32))
    mg = oracle.neighbor_merge(poses, None, srt, P)
    psi = rng.normal(size=(n, 6)) * 0.1
    return poses, P, mg, psi


def test_preconditioned_repulsion_limits(oracle):
    """The preconditioned reading reduces to Eq. 6 as printed when every
    damped Hessian is the identity, scales the repulsion by 1/s when it is s I,
    and leaves the attraction (sum_j k_ij psi_j) untouched."""
    poses, P, mg, psi = _all_pairs_case(oracle)
    n = len(poses)
    phi_lit, _ = oracle.svgd(poses, mg["ids"], mg["k"], mg["d"], psi, P)
    # H with H + lambda diag H + eps I = I
    h = (1.0 - P.eps_damp) / (1.0 + P.lam)
    H = np.zeros((n, 21))
    H[:, [0, 6, 11, 15, 18, 20]] = h
    pinv = oracle.svgd_precond_matrices(H, np.ones(n, np.int32), P)
    assert np.allclose(pinv, np.eye(6), atol=1e-14)
    phi_id, _ = oracle.svgd(poses, mg["ids"], mg["k"], mg["d"], psi, P, pinv)
    assert np.allclose(phi_id, phi_lit, atol=1e-14)
    # the attraction alone: no repulsion (zero preconditioner)
    phi_att, _ = oracle.svgd(poses, mg["ids"], mg["k"], mg["d"], psi, P, np.zeros((n, 6, 6)))
    for s in (0.5, 4.0):
        phi_s, _ = oracle.svgd(poses, mg["ids"], mg["k"], mg["d"], psi, P, np.broadcast_to(np.eye(6) / s, (n, 6, 6)))
        assert np.allclose(phi_s - phi_att, (phi_lit - phi_att) / s, atol=1e-14)
    # particles without a Gauss-Newton step get no repulsion
    pinv0 = oracle.svgd_precond_matrices(H, np.zeros(n, np.int32), P)
    assert not pinv0.any()


@pytest.mark.parametrize("scale", [1e-2, 3e-3])
def test_kernel_gradient_fd(oracle, scale):
    # grad_{T_j} k(T_i, T_j) for a right perturbation T_j exp(h e_a) equals
    # -2 k W d_ij up to O(|d|^2) relative (Eq. 6, first order in d).
    rng = np.random.default_rng(2)
    W = np.array([5.0] * 3 + [2.5] * 3)
    Ti = mat(np.concatenate([Rotation.random(random_state=3).as_quat(), rng.normal(size=3)]))
    d0 = rng.normal(size=6)
    d0 *= scale / np.linalg.norm(d0)
    Tj = Ti @ expm(hat(d0))
    k = lambda T: np.exp(-(W * vee(np.real(logm(np.linalg.inv(Ti) @ T))) ** 2).sum())
    h = 1e-7
    g = np.array([(k(Tj @ expm(hat(h * e))) - k(Tj @ expm(hat(-h * e)))) / (2 * h) for e in np.eye(6)])
    pred = -2 * k(Tj) * W * d0
    assert np.linalg.norm(g - pred) <= 3 * scale * np.linalg.norm(pred) + 1e-9


def test_posterior_ring_golden(oracle):
    g = json.load(open(os.path.join(GOLDEN, "posterior_ring4.json")))
    ids = np.array([[i, (i - 1) % 4, (i + 1) % 4] for i in range(4)], np.int32)
    kk = np.ones((4, 3))
    loglik = np.log(np.array(g["p_init"]) + 1e-300)
    for it, key in ((1, "after_1"), (2, "after_2")):
        p0, p, best = oracle.posterior(None, loglik, ids, kk, it)
        assert np.allclose(p0, g["p_init"], atol=1e-15)
        assert np.allclose(p, g[key], atol=1e-15)
    # ten sweeps: the doubly stochastic averaging matrix to the 10th power
    M = np.zeros((4, 4))
    for i in range(4):
        M[i, ids[i]] = 1 / 3
    p0, p, best = oracle.posterior(None, loglik, ids, kk, 10)
    assert np.allclose(p, np.linalg.matrix_power(M, 10) @ np.array(g["p_init"]), atol=1e-15)
    assert best == 0


def test_posterior_fixed_points_and_log_domain(oracle):
    rng = np.random.default_rng(3)
    n, K = 200, 6
    ids = rng.integers(0, n, (n, K)).astype(np.int32)
    ids[:, 0] = np.arange(n)
    ids[rng.random((n, K)) < 0.2] = -1
    ids[:, 0] = np.arange(n)
    kk = rng.uniform(0.1, 1.0, (n, K)); kk[:, 0] = 1.0
    p0, p, best = oracle.posterior(np.full(n, -3.0), np.full(n, -1e4), ids, kk, 10)
    assert np.allclose(p, 1.0 / n, rtol=1e-12)                    # uniform is a fixed point
    # exact ties (lists = {self}, equal log-likelihoods): the smaller index wins
    solo = np.full((n, 1), -1, np.int32); solo[:, 0] = np.arange(n)
    llt = np.full(n, -50.0); llt[[17, 9, 120]] = -1.0
    _, pt, bt = oracle.posterior(None, llt, solo, np.ones((n, 1)), 10)
    assert pt[17] == pt[9] == pt[120] and bt == 9
    ll = np.zeros(n); ll[5] = -1e4 + 2.0; ll[:] = -1e4; ll[5] += 2.0; ll[7] += 1.0
    p0, _, _ = oracle.posterior(None, ll, ids, kk, 0)
    assert np.isclose(p0[5] / p0[7], np.e) and np.isclose(p0[5] / p0[0], np.e ** 2)
    p0, p, best = oracle.posterior(None, ll, ids, kk, 10)
    assert abs(p.sum() - 1) < 1e-12


def test_cholesky_and_prediction_without_noise(oracle):
    rng = np.random.default_rng(4)
    A = rng.normal(size=(6, 6)); S = A @ A.T + 0.1 * np.eye(6)
    assert np.allclose(oracle.cholesky6(S), np.linalg.cholesky(S), atol=1e-12)
    S2 = np.diag([0.1, 0, 0.2, 0, 0, 0.3])
    assert np.allclose(oracle.cholesky6(S2), np.sqrt(S2), atol=1e-15)
    n = 20
    poses = np.concatenate([Rotation.random(n, random_state=5).as_quat(), rng.normal(size=(n, 3))], 1).astype(np.float32)
    D = np.eye(4); D[:3, :3] = Rotation.from_rotvec([0.1, -0.05, 0.2]).as_matrix(); D[:3, 3] = [1.0, 0.2, -0.3]
    out, delta = oracle.predict(poses, D, np.zeros((6, 6)), 4, 0, want_delta=True)
    assert np.all(delta == 0)
    for i in range(n):
        assert np.allclose(mat(out[i]), mat(poses[i]) @ D, atol=1e-12)


def test_prediction_noise_statistics(oracle):
    n = 20000
    poses = np.tile(np.array([0, 0, 0, 1, 0, 0, 0], np.float32), (n, 1))
    S = np.diag([0.01 ** 2] * 3 + [0.05 ** 2] * 3)
    S[3, 4] = S[4, 3] = 0.5 * 0.05 * 0.05
    out, delta = oracle.predict(poses, np.eye(4), S, 4, 7, want_delta=True)
    C = np.cov(delta.T)
    assert np.allclose(C, S, atol=0.06 * S.max())
    for i in range(0, n, 997):        # T exp(delta)
        assert np.allclose(mat(out[i]), expm(hat(delta[i])), atol=1e-12)
    z = np.array([oracle.predict_noise(i, 4, 7) for i in range(4000)]).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_philox_stream_properties(oracle):
    out = np.array([oracle.philox([i, 0, 0, 0], [4, 0]) for i in range(4000)])
    assert len(np.unique(out[:, 0])) == 4000                     # distinct counters, distinct words
    u = (out.astype(np.float64).ravel() + 0.5) / 2 ** 32
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    bits = np.unpackbits(out.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.01
    a = oracle.philox([1, 2, 3, 4], [5, 6]); b = oracle.philox([1, 2, 3, 4], [5, 7])
    assert not np.array_equal(a, b)
    u53 = np.array([oracle.lib().or_uniform53(4, 0, 2, k) for k in range(4000)])
    assert u53.min() >= 0 and u53.max() < 1 and stats.kstest(u53, "uniform").pvalue > 1e-3


def test_uniform_init(oracle):
    n = 20000
    lo = np.array([-5, -5, 0, -np.deg2rad(5), -np.deg2rad(5), -np.pi])
    hi = np.array([5, 5, 2, np.deg2rad(5), np.deg2rad(5), np.pi])
    out = oracle.init_uniform(n, lo, hi, 3)
    assert np.all(out[:, 4:] >= lo[:3]) and np.all(out[:, 4:] <= hi[:3])
    ypr = Rotation.from_quat(out[:, :4]).as_euler("ZYX")
    assert np.all(np.abs(ypr[:, 1]) <= np.deg2rad(5) + 1e-9) and np.all(np.abs(ypr[:, 2]) <= np.deg2rad(5) + 1e-9)
    assert stats.kstest((ypr[:, 0] + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-3
    full = oracle.init_uniform(n, [-1, -1, -1, -np.pi, -np.pi, -np.pi], [1, 1, 1, np.pi, np.pi, np.pi], 3)
    R = Rotation.from_quat(full[:, :4]).as_matrix().mean(0)
    assert np.abs(R).max() < 0.03            # Haar measure: E[R] = 0


def test_philox_known_answers(oracle):
    """Philox-4x32-10 against the known-answer vectors its authors publish
    (tests/golden/philox4x32_10_kat.json): a swapped output word, a wrong
    multiplier or key schedule fails here, which statistics would not show."""
    import json
    import os
    kat = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(w, 16) for w in v["ctr"]]
        key = [int(w, 16) for w in v["key"]]
        out = [int(w) for w in oracle.philox(ctr, key)]
        assert out == [int(w, 16) for w in v["out"]], v


def test_posterior_floor(oracle):
    """The floor of the initial posterior (Sec. III-D prior; the reading that
    keeps exp(l - max l) >= exp(-floor)): without it a particle far below the
    best has an exact zero posterior, its log prior is -inf at the next step
    and it can never win again; with it, its posterior is exp(-floor) relative
    to the best, and a decisive likelihood at the next step makes it the
    representative state."""
    n = 4
    ids = np.arange(n, dtype=np.int32)[:, None]          # lists = {self}: no smoothing
    kk = np.ones((n, 1))
    ll1 = np.array([0.0, -1e5, -50.0, -800.0])
    for floor in (0.0, 700.0):
        p0, p, best = oracle.posterior(None, ll1, ids, kk, 0, floor)
        assert best == 0
        if floor == 0.0:
            assert p[1] == 0.0 and p[3] == 0.0
        else:
            # exp(max(l - max l, -floor)) / sum, term by term
            w = np.exp(np.maximum(ll1 - 0.0, -floor))
            assert np.allclose(p, w / w.sum(), rtol=1e-14, atol=0)
            assert p[1] == p[3] > 0
        with np.errstate(divide="ignore"):
            prior2 = np.log(p)
        # the next step: particle 1 now explains the scan, particle 0 does not
        ll2 = np.array([-1000.0, 0.0, -2000.0, -900.0])
        _, p2, best2 = oracle.posterior(prior2, ll2, ids, kk, 0, floor)
        assert best2 == (0 if floor == 0.0 else 1)
    # the floor is relative to the best particle, so it does not depend on an offset of l
    a = oracle.posterior(None, ll1 + 1234.5, ids, kk, 0, 700.0)[1]
    b = oracle.posterior(None, ll1, ids, kk, 0, 700.0)[1]
    assert np.allclose(a, b, rtol=1e-12, atol=0)
