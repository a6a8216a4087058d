"""Pins of the oracle's point Gaussians (Sec. III-C, GICP model of each point)
and its NNF (Sec. III-C, nearest neighbour field): closed forms on planes, the
library eigen-solver, and brute force written independently in numpy with the
same FP32 decision sequence."""
import numpy as np
import pytest

from paper_2404_16370_gb300 import synth


def knn_numpy(pts, r, k):
    """Brute-force radius-limited kNN; distances by the FP32 sequence
    ((dx*dx + dy*dy) + dz*dz), ties to the smaller index."""
    pts = pts.astype(np.float32)
    out = []
    for i in range(len(pts)):
        d = pts - pts[i]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        r2 = np.float32(r) * np.float32(r)
        idx = np.nonzero(d2 <= r2)[0]
        order = np.lexsort((idx, d2[idx]))
        out.append(idx[order][:k])
    return out


def test_sym3_eigh_matches_numpy(oracle):
    rng = np.random.default_rng(0)
    for _ in range(200):
        A = rng.normal(size=(3, 3))
        A = A @ A.T * rng.uniform(1e-3, 10)
        w, V = oracle.sym3_eigh(A)
        w2, V2 = np.linalg.eigh(A)
        assert np.allclose(w, w2, rtol=1e-12, atol=1e-14 * np.abs(w2).max())
        for c in range(3):
            assert min(np.abs(V[:, c] - V2[:, c]).max(), np.abs(V[:, c] + V2[:, c]).max()) < 1e-9
        assert np.allclose(V @ np.diag(w) @ V.T, A, atol=1e-12 * np.abs(A).max())


def test_plane_normal_closed_form(oracle):
    # points of the plane z = 0.3 x - 0.2 y + 1: every neighbourhood is planar, so the
    # normal is (-0.3, 0.2, 1)/|.| and the smallest covariance eigenvalue is 0.
    g = np.stack(np.meshgrid(np.arange(-10, 11) * 0.1, np.arange(-10, 11) * 0.1), -1).reshape(-1, 2)
    pts = np.concatenate([g, (0.3 * g[:, 0] - 0.2 * g[:, 1] + 1.0)[:, None]], -1).astype(np.float32)
    n, valid, _, covs = oracle.point_normals(pts, 0.35, 10, 5, want_covs=True)
    assert valid.all()
    ref = np.array([-0.3, 0.2, 1.0]) / np.linalg.norm([-0.3, 0.2, 1.0])
    assert np.abs(np.abs(n @ ref) - 1).max() < 1e-6      # FP32 inputs: the plane is exact to ~1e-7
    w = np.linalg.eigvalsh(covs.reshape(-1, 3, 3))
    assert np.abs(w[:, 0]).max() < 1e-12


def test_neighbourhoods_and_covariances_brute_force(oracle):
    rng = np.random.default_rng(1)
    pts = (rng.normal(size=(600, 3)) * [1.0, 1.0, 0.2]).astype(np.float32)
    pts[:20] += 30.0                                   # an isolated cluster of 20 points
    pts[20] = [50, 50, 50]                             # a lone point -> invalid
    r, k, kmin = 0.6, 10, 5
    ref = knn_numpy(pts, r, k)
    for brute in (True, False):
        n, valid, nbrs, covs = oracle.point_normals(pts, r, k, kmin, brute=brute, want_nbrs=True, want_covs=True)
        for i in range(len(pts)):
            got = nbrs[i][nbrs[i] >= 0]
            assert np.array_equal(got, ref[i]), i
            assert valid[i] == (len(ref[i]) >= kmin)
            if valid[i]:
                C = np.cov(pts[ref[i]].astype(np.float64).T, bias=True)
                assert np.allclose(covs[i].reshape(3, 3), C, atol=1e-12)
                w, V = np.linalg.eigh(C)
                assert abs(abs(n[i] @ V[:, 0]) - 1) < 1e-8
    assert not valid[20]


def test_nnf_brute_force_all_voxels(oracle):
    rng = np.random.default_rng(2)
    pts = rng.uniform(-0.6, 0.6, (150, 3)).astype(np.float32)
    valid = np.ones(150, np.uint8)
    valid[::7] = 0                                        # invalid map points never qualify
    P = oracle.Params(res=0.1, r_max=0.25)
    m = oracle.OracleMap(pts, P, normals=np.tile([0, 0, 1.0], (150, 1)), valid=valid)
    o, dims, inv_res, off = m.geometry()
    # (D4) geometry, recomputed in numpy FP32
    vp = pts[valid.astype(bool)]
    lo, hi = vp.min(0), vp.max(0)
    r32, res32 = np.float32(0.25), np.float32(0.1)
    inv32 = np.float32(1) / res32
    assert np.array_equal(o, lo - r32)
    assert np.array_equal(dims, (np.floor(((hi + r32) - (lo - r32)) * inv32) + 1).astype(np.int32))
    vox = np.stack(np.meshgrid(*[np.arange(-1, d + 1) for d in dims], indexing="ij"), -1).reshape(-1, 3)
    got_grid = m.nnf(vox)
    got_brute = m.nnf(vox, brute=True)
    assert np.array_equal(got_grid, got_brute)
    # independent numpy brute force with (D6) centres and (D3) distances
    ref = np.full(len(vox), -1, np.int32)
    inside = np.all((vox >= 0) & (vox < dims), axis=1)
    cen = o + ((vox.astype(np.float32) + np.float32(0.5)) * res32)
    vidx = np.nonzero(valid)[0]
    r2 = r32 * r32
    for a in np.nonzero(inside)[0]:
        d = pts[vidx] - cen[a]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        ok = d2 <= r2
        if ok.any():
            cand = np.nonzero(ok)[0]
            best = cand[np.lexsort((vidx[cand], d2[cand]))[0]]
            ref[a] = vidx[best]
    assert np.array_equal(got_grid, ref)
    assert (ref >= 0).sum() > 100 and (ref[inside] < 0).sum() > 0


def test_map_normals_on_box_room(oracle):
    # walls of the room: normals along the axes for points away from edges
    room = synth.box_room(1, n_map=6000, n_boxes=0)
    n, valid, _, _ = oracle.point_normals(room.map_points, 0.8, 10, 5)
    p = room.map_points
    floor = (np.abs(p[:, 2]) < 1e-5) & (np.abs(p[:, 0]) < 4) & (np.abs(p[:, 1]) < 4)
    wall = (np.abs(p[:, 0] - 5) < 1e-5) & (p[:, 2] > 0.8) & (p[:, 2] < 2.2) & (np.abs(p[:, 1]) < 4)
    assert valid[floor].all() and valid[wall].all()
    assert np.abs(np.abs(n[floor, 2]) - 1).max() < 1e-9
    assert np.abs(np.abs(n[wall, 0]) - 1).max() < 1e-9
