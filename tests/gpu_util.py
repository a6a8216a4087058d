"""Helpers of the GPU parity tests: comparisons against the oracle with the
tolerances the tests state, and SE(3) distances between pose arrays."""
import numpy as np
from scipy.spatial.transform import Rotation


def pose_error(a, b):
    """(rotation angle, translation distance) between (n,7) pose arrays."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ra = Rotation.from_quat(a[:, :4] / np.linalg.norm(a[:, :4], axis=1, keepdims=True))
    rb = Rotation.from_quat(b[:, :4] / np.linalg.norm(b[:, :4], axis=1, keepdims=True))
    ang = (ra.inv() * rb).magnitude()
    return ang, np.linalg.norm(a[:, 4:] - b[:, 4:], axis=1)


def sum_tolerance(ref_abs, rel=1e-4, floor=1e-6):
    """1e-4 of the sum of term magnitudes (the rounding scale of an FP32 sum)."""
    return rel * ref_abs + floor


def report(name, err, tol):
    bad = err > tol
    if bad.any():
        k = np.argmax(err - tol)
        return f"{name}: {bad.sum()} entries over tolerance; worst err {err.flat[k]:.3g} tol {tol.flat[k]:.3g}"
    return ""


def check_sums(gn, ref, rel=1e-4, floor=1e-6):
    """GPU likelihood sums (n, 29) against the oracle: every particle, with the
    room that ambiguous inlier decisions give (a pair within 1e-4 of c_max may
    fall either way in FP32): |gpu - ref| <= rel * sum|terms| + sum over
    ambiguous pairs of |term|, and |inliers - ref| <= ambiguous pairs."""
    d_in = np.abs(gn[:, 28].astype(np.int64) - ref["n_in"])
    assert np.all(d_in <= ref["amb"]), f"inlier counts: {np.sum(d_in > ref['amb'])} particles off"
    got = gn[:, :28].astype(np.float64)
    want = np.concatenate([ref["H"], ref["b"], ref["loglik"][:, None]], 1)
    tol = rel * ref["absum"] + ref["ambabs"] + floor
    return report("H/b/loglik", np.abs(got - want), tol)


def visit_order(sorted_ids, t, info):
    """The likelihood's visiting order as the library defines it: particles by
    the Morton code of their position's cell (cubes of 2^s NNF voxels, s the
    smallest shift leaving at most 32 cubes along every axis; positions clamped
    to the grid, NaN to cell 0), stable over the LSH order. The voxel
    coordinate is a float32 product and sum, as in the kernel."""
    t = np.asarray(t, np.float32)
    inv = np.float32(info["inv_res"])
    off = np.asarray(info["off"], np.float32)
    dims = np.asarray(info["dims"], np.int64)
    s = 0
    while (int(dims.max()) - 1) >> s >= 32:
        s += 1
    key = np.zeros(len(t), np.int64)
    with np.errstate(invalid="ignore"):
        for a in range(3):
            f = t[:, a] * inv + off[a]
            v = np.where(f >= 0, np.floor(np.minimum(f, np.float32(dims[a] - 1))), 0).astype(np.int64)
            c = v >> s
            for b in range(5):
                key |= ((c >> b) & 1) << (3 * b + a)
    sid = np.asarray(sorted_ids, np.int64)
    return sid[np.argsort(key[sid], kind="stable")]
