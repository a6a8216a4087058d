"""Pins of the oracle's LSH keys (Eq. 9, 10), bucketing and neighbour-list
refinement (Algorithm 1): the integer hash computed by hand, alpha -> 0
degenerating to one bucket, numpy's stable argsort, exact k-NN by brute force
over all particles, and the bucket window on a hand-built example."""
import numpy as np
import pytest
from scipy.linalg import logm
from scipy.spatial.transform import Rotation

P_HASH = [73856093, 19349663, 83492791, 2654435761, 805459861, 3674653429]


def test_hash_multipliers_are_odd():
    # odd multipliers make c -> c * P mod 2^32 a bijection of each component
    assert all(p % 2 == 1 for p in P_HASH)


def test_key_by_hand(oracle):
    # T_LSH = identity, alpha = 1, particles with R = I: log(T) = (0, 0, 0, t) and
    # zeta = W t + delta; with delta = 0.5 the floors are known exactly.
    P = oracle.Params(sigma_r=5.0, sigma_t=2.5, alpha=1.0, nb_log2=32)
    ts = np.array([[0.0, 0.0, 0.0], [1.0, -2.0, 3.0], [-7.2, 0.33, 100.1], [-0.1, -0.1, -0.1]])
    poses = np.concatenate([np.tile([0, 0, 0, 1.0], (len(ts), 1)), ts], 1).astype(np.float32)
    delta = np.full(6, 0.5)
    out = oracle.lsh_keys(poses, [0, 0, 0, 1.0], [0, 0, 0], delta, P, want_zeta=True)
    for i, t in enumerate(poses[:, 4:].astype(np.float64)):
        zeta = np.concatenate([np.full(3, 0.5), 2.5 * t + 0.5])
        assert np.allclose(out["zeta"][i], zeta, atol=1e-12)
        key = 0
        for c, p in zip(np.floor(zeta).astype(np.int64), P_HASH):
            key ^= (int(c) * p) % (1 << 32)
        assert int(out["keys"][i]) == key
        assert int(out["buckets"][i]) == key
    P12 = oracle.Params(alpha=1.0, nb_log2=12)
    out12 = oracle.lsh_keys(poses, [0, 0, 0, 1.0], [0, 0, 0], delta, P12)
    assert np.array_equal(out12["buckets"], out["keys"] & 4095)


def test_alpha_zero_is_one_bucket_and_flags(oracle):
    rng = np.random.default_rng(0)
    n = 300
    poses = np.concatenate([Rotation.random(n, random_state=1).as_quat(), rng.normal(size=(n, 3)) * 5], 1).astype(np.float32)
    P = oracle.Params(alpha=0.0, nb_log2=10)
    out = oracle.lsh_keys(poses, [0, 0, 0, 1.0], [0, 0, 0], [0.3, 1.7, -0.2, 2.5, 0.1, -3.9], P)
    assert len(np.unique(out["keys"])) == 1 and not out["flags"].any()
    out = oracle.lsh_keys(poses, [0, 0, 0, 1.0], [0, 0, 0], [0.3, 1.7, -0.2, 2.0, 0.1, -3.9], P)
    assert out["flags"].all()          # zeta_4 = 2.0 exactly: on a cell boundary


def test_lsh_draw_distribution(oracle):
    lo, hi = np.array([-5.0, -5, 0]), np.array([5.0, 5, 3])
    D, T, Q = [], [], []
    for s in range(2000):
        q, t, d = oracle.lsh_draw(4, s, lo, hi, 0.5)
        assert abs(np.linalg.norm(q) - 1) < 1e-12 and np.all(t >= lo) and np.all(t <= hi)
        D.append(d); T.append(t); Q.append(q)
    D = np.array(D)
    assert np.abs(D.mean(0)).max() < 0.05 and np.abs(D.std(0) - 0.5).max() < 0.05
    # uniform rotations: E[R] = 0
    Rm = Rotation.from_quat(np.array(Q)).as_matrix().mean(0)
    assert np.abs(Rm).max() < 0.08
    q0, t0, d0 = oracle.lsh_draw(4, 0, lo, hi, 0.5)
    q1, t1, d1 = oracle.lsh_draw(5, 0, lo, hi, 0.5)
    assert not np.allclose(d0, d1)


def test_bucket_sort_matches_stable_argsort(oracle):
    rng = np.random.default_rng(3)
    b = rng.integers(0, 50, 5000).astype(np.uint32)
    s = oracle.bucket_sort(b)
    ref = np.argsort(b, kind="stable")
    assert np.array_equal(s["sorted_ids"], ref)
    assert np.array_equal(s["rank"][ref], np.arange(5000))
    starts = np.searchsorted(b[ref], b, side="left")
    ends = np.searchsorted(b[ref], b, side="right")
    assert np.array_equal(s["seg_lo"], starts) and np.array_equal(s["seg_hi"], ends)


def _pose_mats(poses):
    Ts = []
    for p in poses.astype(np.float64):
        T = np.eye(4)
        T[:3, :3] = Rotation.from_quat(p[:4] / np.linalg.norm(p[:4])).as_matrix()
        T[:3, 3] = p[4:]
        Ts.append(T)
    return Ts


def _vee(M):
    return np.array([M[2, 1], M[0, 2], M[1, 0], M[0, 3], M[1, 3], M[2, 3]])


def test_exact_knn_when_window_covers_everything(oracle):
    # alpha = 0 puts every particle in one bucket; with C >= N every particle is a
    # candidate, so the list must be the exact K nearest under s (Eq. 7, 8).
    rng = np.random.default_rng(4)
    n, K = 60, 8
    rot = Rotation.from_rotvec(rng.normal(size=(n, 3)) * 0.3)
    poses = np.concatenate([rot.as_quat(), rng.normal(size=(n, 3))], 1).astype(np.float32)
    P = oracle.Params(alpha=0.0, K=K, C=n + 4, nb_log2=6)
    keys = oracle.lsh_keys(poses, [0, 0, 0, 1.0], [0, 0, 0], np.full(6, 0.5), P)
    srt = oracle.bucket_sort(keys["buckets"])
    mg = oracle.neighbor_merge(poses, None, srt, P)
    Ts = _pose_mats(poses)
    W = np.array([5.0] * 3 + [2.5] * 3)
    for i in range(n):
        s = np.array([W @ _vee(np.real(logm(np.linalg.inv(Ts[i]) @ Ts[j]))) ** 2 if False else
                      (W * _vee(np.real(logm(np.linalg.inv(Ts[i]) @ Ts[j]))) ** 2).sum() for j in range(n)])
        s[i] = -1
        order = np.lexsort((np.arange(n), s))[:K]
        assert mg["ids"][i, 0] == i and mg["k"][i, 0] == 1.0
        if mg["flags"][i]:
            continue
        assert set(mg["ids"][i]) == set(order), i
        got = mg["ids"][i, 1:]
        assert np.allclose(mg["k"][i, 1:], np.exp(-s[got]), rtol=1e-7)
        assert np.all(np.diff(s[got]) >= -1e-12)       # stored sorted by s


def test_window_and_old_list_on_hand_example(oracle):
    # 10 particles on a line along x (identity rotations) in one bucket.
    n, K, C = 10, 5, 4
    poses = np.zeros((n, 7), np.float32)
    poses[:, 3] = 1
    poses[:, 4] = np.arange(n) * 1.0
    P = oracle.Params(alpha=0.0, K=K, C=C, nb_log2=4)
    srt = oracle.bucket_sort(np.zeros(n, np.uint32))
    mg = oracle.neighbor_merge(poses, None, srt, P)
    for i in range(n):
        s = min(max(i - C // 2, 0), n - C)
        window = set(range(s, s + C)) - {i}
        assert set(mg["ids"][i][mg["ids"][i] >= 0]) == window | {i}
    # an old neighbour closer than the window members survives the merge
    old = np.full((n, K), -1, np.int32)
    old[:, 0] = np.arange(n)
    old[9, 1] = 8
    srt2 = dict(srt)
    srt2["sorted_ids"] = np.array([9, 0, 1, 2, 3, 4, 5, 6, 7, 8], np.int32)
    srt2["rank"] = np.argsort(srt2["sorted_ids"]).astype(np.int32)
    mg2 = oracle.neighbor_merge(poses, old, srt2, P)
    assert 8 in mg2["ids"][9]
    assert mg2["ids"][9, 1] == 8            # nearest first


def test_kernel_values_symmetric(oracle):
    rng = np.random.default_rng(5)
    n = 40
    poses = np.concatenate([Rotation.random(n, random_state=2).as_quat(), rng.normal(size=(n, 3))], 1).astype(np.float32)
    W = np.array([5.0] * 3 + [2.5] * 3)
    for i in range(n):
        for j in range(i + 1, n):
            dij = oracle.relative_log(poses[i], poses[j])
            dji = oracle.relative_log(poses[j], poses[i])
            if np.linalg.norm(dij[:3]) < np.pi - 1e-6:
                assert abs((W * dij ** 2).sum() - (W * dji ** 2).sum()) < 1e-10 * max(1, (W * dij ** 2).sum())
