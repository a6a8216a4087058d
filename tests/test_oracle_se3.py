"""Pins of the oracle's SE(3) maps (Sec. III-B Eq. 1, Sec. III-C Eq. 5 and 8)
against library routines: scipy.linalg.expm / logm of the 4x4 twist matrix and
scipy's rotation conversions."""
import numpy as np
import pytest
from scipy.linalg import expm, logm
from scipy.spatial.transform import Rotation


def hat(xi):
    w, v = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def vee(M):
    return np.array([M[2, 1], M[0, 2], M[1, 0], M[0, 3], M[1, 3], M[2, 3]])


def mat(q, t):
    T = np.eye(4)
    T[:3, :3] = Rotation.from_quat(q).as_matrix()
    T[:3, 3] = t
    return T


@pytest.mark.parametrize("scale", [1e-9, 1e-6, 1e-3, 0.3, 1.5, 3.0])
def test_exp_matches_expm(oracle, scale):
    rng = np.random.default_rng(int(scale * 1e9) % 1000)
    for _ in range(20):
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        xi = np.concatenate([w, rng.normal(size=3) * 2])
        q, t = oracle.se3_exp(xi)
        T = expm(hat(xi))
        assert np.allclose(mat(q, t), T, atol=1e-12, rtol=0)
        assert abs(np.linalg.norm(q) - 1) < 1e-14


@pytest.mark.parametrize("scale", [1e-8, 1e-4, 0.5, 2.5])
def test_log_matches_logm_and_roundtrip(oracle, scale):
    rng = np.random.default_rng(7)
    for _ in range(20):
        w = rng.normal(size=3)
        w = w / np.linalg.norm(w) * scale
        xi = np.concatenate([w, rng.normal(size=3)])
        T = expm(hat(xi))
        q = Rotation.from_matrix(T[:3, :3]).as_quat()
        lg = oracle.se3_log(q, T[:3, 3])
        assert np.allclose(lg, xi, atol=1e-11)
        assert np.allclose(lg, vee(np.real(logm(T))), atol=1e-8)
        q2, t2 = oracle.se3_exp(lg)
        assert np.allclose(mat(q2, t2), T, atol=1e-12)


def test_pure_translation_and_rotation(oracle):
    # omega = 0: exp is a pure translation
    q, t = oracle.se3_exp([0, 0, 0, 1.0, -2.0, 3.0])
    assert np.allclose(q, [0, 0, 0, 1]) and np.allclose(t, [1, -2, 3])
    # rotation by 90 deg about z
    q, t = oracle.se3_exp([0, 0, np.pi / 2, 0, 0, 0])
    R = oracle.quat_to_rot(q)
    assert np.allclose(R, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)


def test_quat_rot_conversions(oracle):
    rng = np.random.default_rng(3)
    for q in Rotation.random(50, random_state=4).as_quat():
        assert np.allclose(oracle.quat_to_rot(q), Rotation.from_quat(q).as_matrix(), atol=1e-14)
        q2 = oracle.rot_to_quat(Rotation.from_quat(q).as_matrix())
        assert min(np.abs(q2 - q).max(), np.abs(q2 + q).max()) < 1e-13
    del rng


def test_relative_log_is_log_of_relative_transform(oracle):
    rng = np.random.default_rng(5)
    for _ in range(50):
        qi, qj = Rotation.random(2, random_state=rng.integers(1 << 30)).as_quat()
        ti, tj = rng.normal(size=3) * 10, rng.normal(size=3) * 10
        pi = np.concatenate([qi, ti]).astype(np.float32)
        pj = np.concatenate([qj, tj]).astype(np.float32)
        d = oracle.relative_log(pi, pj)
        Ti = mat(pi[:4].astype(np.float64) / np.linalg.norm(pi[:4].astype(np.float64)), pi[4:].astype(np.float64))
        Tj = mat(pj[:4].astype(np.float64) / np.linalg.norm(pj[:4].astype(np.float64)), pj[4:].astype(np.float64))
        rel = np.linalg.inv(Ti) @ Tj
        if np.linalg.norm(d[:3]) < np.pi - 1e-3:
            assert np.allclose(d, vee(np.real(logm(rel))), atol=1e-8)
        # antisymmetry: d_ji = -d_ij, so s_ij = s_ji (Eq. 7 is symmetric)
        dji = oracle.relative_log(pj, pi)
        if np.linalg.norm(d[:3]) < np.pi - 1e-6:
            assert np.allclose(dji, -d, atol=1e-11)


@pytest.mark.parametrize("theta", [1e-6, 1e-4, 1e-3, 5e-3, 1e-2, 2e-2, 0.1])
def test_log_small_angle_large_translation(oracle, theta):
    # the translation part of log (V^-1 t) must stay accurate where
    # 1 - cos(theta) cancels: LSH floors (Eq. 10) depend on it at 1e-9
    xi = np.array([theta, 0.3 * theta, -0.2 * theta, 100.0, 50.0, -30.0])
    T = expm(hat(xi))
    q = Rotation.from_matrix(T[:3, :3]).as_quat()
    assert np.abs(oracle.se3_log(q, T[:3, 3]) - xi).max() < 1e-12
