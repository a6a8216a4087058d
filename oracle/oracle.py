"""Python driver for the FP64 CPU oracle (oracle.cpp).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference arm are the only callers. The product path (the CUDA
library and its binding) never imports this module, and this module never
imports the product package.

The stage functions mirror the steps of one filter step of the paper, in its
order (Table II rows: neighbour list update, likelihood evaluation, particle
state update, posterior probability update), preceded by the prediction of
Sec. III-B. ``OracleFilter.step`` chains them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, OpenMP, no FP contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB)
            _declare(_lib)
    return _lib


_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double
_F = C.c_float
_INT = C.c_int
_U64 = C.c_uint64
_U32 = C.c_uint32


def _declare(L):
    L.or_philox4x32_10.argtypes = [_P, _P, _P]
    L.or_uniform53.argtypes = [_U64, _U64, _U32, _U32]
    L.or_uniform53.restype = _D
    L.or_quat_to_rot.argtypes = [_P, _P]
    L.or_rot_to_quat.argtypes = [_P, _P]
    L.or_se3_exp.argtypes = [_P, _P, _P]
    L.or_se3_log.argtypes = [_P, _P, _P]
    L.or_relative_log.argtypes = [_P, _P, _P]
    L.or_sym3_eigh.argtypes = [_P, _P, _P]
    L.or_point_normals.argtypes = [_P, _I64, _F, _INT, _INT, _INT, _P, _P, _P, _P, _INT]
    L.or_map_create.argtypes = [_P, _I64, _P, _P, _F, _F]
    L.or_map_create.restype = _P
    L.or_map_destroy.argtypes = [_P]
    L.or_map_geometry.argtypes = [_P, _P, _P, _P, _P]
    L.or_map_nnf.argtypes = [_P, _P, _I64, _P, _INT, _INT]
    L.or_voxel_of.argtypes = [_P, _P, _P, _P, _P]
    L.or_likelihood.argtypes = [_P, _P, _I64, _P, _P, _P, _I64, _D, _D, _D, _P, _P, _P, _P, _P, _P, _P, _INT]
    L.or_likelihood_pairs.argtypes = [_P, _P, _P, _P, _P, _I64, _D, _D, _P, _P, _P, _P, _P, _P]
    L.or_gn_solve.argtypes = [_P, _P, _P, _I64, _D, _D, _P, _P]
    L.or_lsh_draw.argtypes = [_U64, _U64, _P, _P, _D, _P, _P, _P]
    L.or_lsh_keys.argtypes = [_P, _I64, _P, _P, _P, _D, _D, _D, _INT, _P, _P, _P, _P]
    L.or_bucket_sort.argtypes = [_P, _I64, _P, _P, _P, _P]
    L.or_neighbor_merge.argtypes = [_P, _I64, _P, _INT, _INT, _P, _P, _P, _P, _D, _D, _D, _P, _I64, _P, _P, _P, _P, _INT]
    L.or_svgd.argtypes = [_P, _I64, _P, _P, _P, _INT, _P, _D, _D, _P, _P, _P]
    L.or_gicp.argtypes = [_P, _P, _P, _I64, _P, _P, _P, _I64, _P, _D, _D, _D, _D, _INT, _D, _P, _P, _P, _P]
    L.or_gicp.restype = _INT
    L.or_posterior.argtypes = [_P, _P, _I64, _P, _P, _INT, _INT, _D, _P, _P, _P]
    L.or_cholesky6.argtypes = [_P, _P]
    L.or_predict_noise.argtypes = [_I64, _U64, _U64, _P]
    L.or_predict.argtypes = [_P, _I64, _P, _P, _U64, _U64, _P, _P]
    L.or_init_uniform.argtypes = [_I64, _P, _P, _U64, _P]


def _p(a):
    # data_as keeps a reference to the array for as long as the pointer object
    # lives (the duration of the call), so temporaries are safe to pass.
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# ---------------------------------------------------------------------------
# Parameters (the oracle's own copy of the readings of the paper; see the
# per-field notes). Two presets: the 10x10x3 m box room and the 200x200x20 m
# outdoor scene.
# ---------------------------------------------------------------------------
@dataclass
class Params:
    res: float = 0.1          # NNF voxel size, m (Sec. III-C: 0.1 indoor, 0.2 outdoor)
    r_max: float = 1.0        # NNF search radius, m
    c_max: float = 9.0        # truncation of the per-point cost
    sigma_r: float = 5.0      # W^K rotation weight, rad^-1 (Eq. 7)
    sigma_t: float = 2.5      # W^K translation weight, m^-1 (Eq. 7)
    alpha: float = 1.0        # LSH scale (Eq. 10)
    lsh_sigma: float = 0.5    # std of delta^LSH (Eq. 10)
    lam: float = 1e-3         # GN damping on diag(H)
    eps_damp: float = 1e-6    # GN damping on I
    eps_cov: float = 1e-3     # GICP normal-direction eigenvalue
    r_cov: float = 1.0        # covariance neighbourhood radius, m
    K: int = 16               # neighbours per particle incl. itself (Sec. III-C: e.g. 20)
    C: int = 16               # bucket window per step
    cov_k: int = 10
    cov_min: int = 5
    post_iters: int = 10      # Eq. 11 iterations (Sec. III-D: e.g. 10)
    nb_log2: int = 12         # log2 of the number of LSH buckets
    seed: int = 4
    svgd_precond: int = 0     # 1: repulsion times (H + lambda diag H + eps I)^-1 (not the printed Eq. 6)
    post_floor: float = 700.0  # floor of the initial posterior exp(l - max l) at exp(-post_floor); 0: none

    @staticmethod
    def box_room(n_particles: int = 4096) -> "Params":
        return Params(res=0.1, r_max=1.0, r_cov=1.0, K=16, C=16,
                      nb_log2=max(1, int(np.ceil(np.log2(max(2, n_particles))))))

    @staticmethod
    def outdoor(n_particles: int = 1 << 20) -> "Params":
        return Params(res=0.2, r_max=2.0, r_cov=2.0, K=32, C=32,
                      nb_log2=max(1, int(np.ceil(np.log2(max(2, n_particles))))))


# ---------------------------------------------------------------------------
# Stage wrappers
# ---------------------------------------------------------------------------
def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(_c(ctr, np.uint32)), _p(_c(key, np.uint32)), _p(out))
    return out


def se3_exp(xi):
    q = np.zeros(4); t = np.zeros(3)
    lib().or_se3_exp(_p(_c(xi, np.float64)), _p(q), _p(t))
    return q, t


def se3_log(q, t):
    xi = np.zeros(6)
    lib().or_se3_log(_p(_c(q, np.float64)), _p(_c(t, np.float64)), _p(xi))
    return xi


def quat_to_rot(q):
    R = np.zeros(9)
    lib().or_quat_to_rot(_p(_c(q, np.float64)), _p(R))
    return R.reshape(3, 3)


def rot_to_quat(R):
    q = np.zeros(4)
    lib().or_rot_to_quat(_p(_c(R, np.float64).reshape(9)), _p(q))
    return q


def relative_log(pi, pj):
    d = np.zeros(6)
    lib().or_relative_log(_p(_c(pi, np.float32)), _p(_c(pj, np.float32)), _p(d))
    return d


def sym3_eigh(A):
    w = np.zeros(3); V = np.zeros(9)
    lib().or_sym3_eigh(_p(_c(A, np.float64).reshape(9)), _p(w), _p(V))
    return w, V.reshape(3, 3)


def point_normals(pts, r_cov, k=10, kmin=5, brute=False, nthreads=0, want_nbrs=False, want_covs=False):
    pts = _c(pts, np.float32)
    n = len(pts)
    normals = np.zeros((n, 3)); valid = np.zeros(n, np.uint8)
    nbrs = np.zeros((n, k), np.int32) if want_nbrs else None
    covs = np.zeros((n, 9)) if want_covs else None
    lib().or_point_normals(_p(pts), n, float(r_cov), k, kmin, int(brute), _p(normals), _p(valid),
                           _p(nbrs), _p(covs), nthreads)
    return normals, valid, nbrs, covs


class OracleMap:
    """Map points, their GICP normals, the NNF geometry and exact NNF queries."""

    def __init__(self, pts, params: Params, nthreads=0, normals=None, valid=None):
        self.pts = _c(pts, np.float32)
        if normals is None:
            normals, valid, _, _ = point_normals(self.pts, params.r_cov, params.cov_k, params.cov_min,
                                                 nthreads=nthreads)
        self.normals = _c(normals, np.float64)
        self.valid = _c(valid, np.uint8)
        self.params = params
        self.h = lib().or_map_create(_p(self.pts), len(self.pts), _p(self.valid), _p(self.normals),
                                     float(params.res), float(params.r_max))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_map_destroy(self.h)
            self.h = None

    def geometry(self):
        o = np.zeros(3, np.float32); d = np.zeros(3, np.int32)
        inv = np.zeros(1, np.float32); off = np.zeros(3, np.float32)
        lib().or_map_geometry(self.h, _p(o), _p(d), _p(inv), _p(off))
        return o, d, float(inv[0]), off

    def nnf(self, vox, brute=False, nthreads=0):
        vox = _c(vox, np.int32).reshape(-1, 3)
        out = np.zeros(len(vox), np.int32)
        lib().or_map_nnf(self.h, _p(vox), len(vox), _p(out), int(brute), nthreads)
        return out

    def voxel_of(self, pose, mu):
        v = np.zeros(3, np.int32); q = np.zeros(3, np.float32)
        lib().or_voxel_of(self.h, _p(_c(pose, np.float32)), _p(_c(mu, np.float32)), _p(v), _p(q))
        return v, q


def likelihood(m: OracleMap, poses, scan, scan_n, scan_valid, params: Params, amb_tol=1e-3, nthreads=0):
    """H (n,21), b (n,6), loglik, n_in, amb (ambiguous inlier decisions),
    absum (n,28): the sum of term magnitudes of each output entry, and ambabs
    (n,28): that sum over the ambiguous pairs (the room either decision has)."""
    poses = _c(poses, np.float32).reshape(-1, 7)
    scan = _c(scan, np.float32).reshape(-1, 3)
    npart = len(poses)
    H = np.zeros((npart, 21)); b = np.zeros((npart, 6)); ll = np.zeros(npart)
    n_in = np.zeros(npart, np.int32); amb = np.zeros(npart, np.int32); absum = np.zeros((npart, 28))
    ambabs = np.zeros((npart, 28))
    lib().or_likelihood(m.h, _p(poses), npart, _p(scan), _p(_c(scan_n, np.float64)),
                        _p(_c(scan_valid, np.uint8)), len(scan), params.c_max, params.eps_cov, amb_tol,
                        _p(H), _p(b), _p(ll), _p(n_in), _p(amb), _p(absum), _p(ambabs), nthreads)
    return dict(H=H, b=b, loglik=ll, n_in=n_in, amb=amb, absum=absum, ambabs=ambabs)


def likelihood_pairs(m: OracleMap, pose, scan, scan_n, scan_valid, params: Params):
    scan = _c(scan, np.float32).reshape(-1, 3)
    ns = len(scan)
    mo = np.zeros(ns, np.int32); e = np.zeros((ns, 3)); om = np.zeros((ns, 3, 3)); J = np.zeros((ns, 3, 6))
    c = np.zeros(ns); inl = np.zeros(ns, np.uint8)
    lib().or_likelihood_pairs(m.h, _p(_c(pose, np.float32)), _p(scan), _p(_c(scan_n, np.float64)),
                              _p(_c(scan_valid, np.uint8)), ns, params.c_max, params.eps_cov,
                              _p(mo), _p(e), _p(om), _p(J), _p(c), _p(inl))
    return dict(m=mo, e=e, omega=om, J=J, c=c, inlier=inl)


H_IDX = np.array([[0, 1, 2, 3, 4, 5], [1, 6, 7, 8, 9, 10], [2, 7, 11, 12, 13, 14],
                  [3, 8, 12, 15, 16, 17], [4, 9, 13, 16, 18, 19], [5, 10, 14, 17, 19, 20]])


def h_full(H21):
    """(n, 21) upper-triangle rows -> (n, 6, 6) symmetric."""
    H21 = np.asarray(H21)
    return H21[..., H_IDX]


def gn_solve(H, b, n_in, params: Params):
    H = _c(H, np.float64); b = _c(b, np.float64); n_in = _c(n_in, np.int32)
    npart = len(n_in)
    psi = np.zeros((npart, 6)); ok = np.zeros(npart, np.int32)
    lib().or_gn_solve(_p(H), _p(b), _p(n_in), npart, params.lam, params.eps_damp, _p(psi), _p(ok))
    return psi, ok


def lsh_draw(seed, step, lo, hi, sigma):
    q = np.zeros(4); t = np.zeros(3); d = np.zeros(6)
    lib().or_lsh_draw(int(seed), int(step), _p(_c(lo, np.float64)), _p(_c(hi, np.float64)), float(sigma),
                      _p(q), _p(t), _p(d))
    return q, t, d


def lsh_keys(poses, q, t, delta, params: Params, want_zeta=False):
    poses = _c(poses, np.float32).reshape(-1, 7)
    npart = len(poses)
    keys = np.zeros(npart, np.uint32); buckets = np.zeros(npart, np.uint32); flags = np.zeros(npart, np.int32)
    zeta = np.zeros((npart, 6)) if want_zeta else None
    lib().or_lsh_keys(_p(poses), npart, _p(_c(q, np.float64)), _p(_c(t, np.float64)), _p(_c(delta, np.float64)),
                      params.alpha, params.sigma_r, params.sigma_t, params.nb_log2,
                      _p(keys), _p(buckets), _p(flags), _p(zeta))
    return dict(keys=keys, buckets=buckets, flags=flags, zeta=zeta)


def bucket_sort(buckets):
    buckets = _c(buckets, np.uint32)
    n = len(buckets)
    sid = np.zeros(n, np.int32); rank = np.zeros(n, np.int32); lo = np.zeros(n, np.int32); hi = np.zeros(n, np.int32)
    lib().or_bucket_sort(_p(buckets), n, _p(sid), _p(rank), _p(lo), _p(hi))
    return dict(sorted_ids=sid, rank=rank, seg_lo=lo, seg_hi=hi)


def neighbor_merge(poses, old_ids, sorting, params: Params, tie_tol=3e-5, nthreads=0, subset=None):
    """New lists of all particles, or of `subset` (rows follow subset)."""
    poses = _c(poses, np.float32).reshape(-1, 7)
    npart, K = len(poses), params.K
    sub = None if subset is None else _c(subset, np.int32)
    nout = npart if sub is None else len(sub)
    ids = np.zeros((nout, K), np.int32); kk = np.zeros((nout, K)); dd = np.zeros((nout, K, 6))
    flags = np.zeros(nout, np.int32)
    lib().or_neighbor_merge(_p(poses), npart, _p(None if old_ids is None else _c(old_ids, np.int32)), K, params.C,
                            _p(_c(sorting["sorted_ids"], np.int32)), _p(_c(sorting["rank"], np.int32)),
                            _p(_c(sorting["seg_lo"], np.int32)), _p(_c(sorting["seg_hi"], np.int32)),
                            params.sigma_r, params.sigma_t, tie_tol, _p(sub), 0 if sub is None else len(sub),
                            _p(ids), _p(kk), _p(dd), _p(flags), nthreads)
    return dict(ids=ids, k=kk, d=dd, flags=flags)


def svgd(poses, ids, kk, dd, psi, params: Params, pinv=None):
    """Eq. 5-6; pinv (n, 6, 6), when given, multiplies each particle's
    repulsive sum (the preconditioned reading, see svgd_precond_matrices)."""
    poses = _c(poses, np.float32).reshape(-1, 7)
    npart = len(poses)
    K = np.asarray(ids).shape[1]
    phi = np.zeros((npart, 6)); out = np.zeros((npart, 7))
    pv = None if pinv is None else _c(pinv, np.float64).reshape(npart, 36)
    lib().or_svgd(_p(poses), npart, _p(_c(ids, np.int32)), _p(_c(kk, np.float64)), _p(_c(dd, np.float64)), K,
                  _p(_c(psi, np.float64)), params.sigma_r, params.sigma_t, _p(pv), _p(phi), _p(out))
    return phi, out


def gicp(src, tgt, params: Params, T0=None, max_iters=30, tol=1e-6, r_corr=None, nthreads=0):
    """Scan-to-scan GICP (Sec. III-B): DeltaT mapping the current scan src into
    the previous scan tgt's frame, the Gauss-Newton H of the last iteration and
    Sigma^DeltaT = H^-1. Point Gaussians from point_normals with the params'
    r_cov / cov_k / cov_min; correspondences within r_corr (default r_max)."""
    src = _c(src, np.float32).reshape(-1, 3)
    tgt = _c(tgt, np.float32).reshape(-1, 3)
    sn, sv, _, _ = point_normals(src, params.r_cov, params.cov_k, params.cov_min, nthreads=nthreads)
    tn, tv, _, _ = point_normals(tgt, params.r_cov, params.cov_k, params.cov_min, nthreads=nthreads)
    T0 = np.eye(4) if T0 is None else _c(T0, np.float64)
    T = np.zeros(16); H = np.zeros(21); nc = np.zeros(1, np.int32); it = np.zeros(1, np.int32)
    lib().or_gicp(_p(src), _p(_c(sn, np.float64)), _p(_c(sv, np.uint8)), len(src), _p(tgt),
                  _p(_c(tn, np.float64)), _p(_c(tv, np.uint8)), len(tgt), _p(_c(T0, np.float64).reshape(16)),
                  float(params.r_max if r_corr is None else r_corr), params.eps_cov, params.lam, params.eps_damp,
                  int(max_iters), float(tol), _p(T), _p(H), _p(nc), _p(it))
    Hm = np.zeros((6, 6))
    Hm[np.triu_indices(6)] = H
    Hm = Hm + np.triu(Hm, 1).T
    with np.errstate(all="ignore"):
        cov = np.linalg.inv(Hm) if nc[0] >= 6 else np.full((6, 6), np.nan)
    return dict(T=T.reshape(4, 4), H=H, cov=cov, n_corr=int(nc[0]), iters=int(it[0]))


def svgd_precond_matrices(H, ok, params: Params):
    """(H + lambda diag H + eps I)^-1 of each particle whose Gauss-Newton step
    was taken (ok), zero otherwise; H given as its 21 upper-triangle entries."""
    H = np.asarray(H, np.float64)
    n = len(H)
    iu = np.triu_indices(6)
    out = np.zeros((n, 6, 6))
    for i in np.nonzero(np.asarray(ok))[0]:
        A = np.zeros((6, 6))
        A[iu] = H[i]
        A = A + np.triu(A, 1).T
        A = A + params.lam * np.diag(np.diag(A)) + params.eps_damp * np.eye(6)
        out[i] = np.linalg.inv(A)
    return out


def posterior(logprior, loglik, ids, kk, iters, floor=0.0):
    """Sec. III-D: initial posterior p_i ~ prior_i p(P | x_i), evaluated as
    exp(l_i - max l) with l = log prior + log-likelihood (floored at
    exp(-floor) when floor > 0), normalised; `iters` Jacobi sweeps of Eq. 11;
    renormalised. Returns (initial posterior, posterior, argmax)."""
    npart = len(loglik)
    K = np.asarray(ids).shape[1]
    p0 = np.zeros(npart); p = np.zeros(npart); best = np.zeros(1, np.int64)
    lib().or_posterior(_p(None if logprior is None else _c(logprior, np.float64)), _p(_c(loglik, np.float64)),
                       npart, _p(_c(ids, np.int32)), _p(_c(kk, np.float64)), K, int(iters), float(floor), _p(p0),
                       _p(p), _p(best))
    return p0, p, int(best[0])


def cholesky6(S):
    L = np.zeros(36)
    lib().or_cholesky6(_p(_c(S, np.float64).reshape(36)), _p(L))
    return L.reshape(6, 6)


def predict_noise(i, seed, step):
    n = np.zeros(6)
    lib().or_predict_noise(int(i), int(seed), int(step), _p(n))
    return n


def predict(poses, odom_T, odom_cov, seed, step, want_delta=False):
    poses = _c(poses, np.float32).reshape(-1, 7)
    npart = len(poses)
    out = np.zeros((npart, 7)); delta = np.zeros((npart, 6)) if want_delta else None
    lib().or_predict(_p(poses), npart, _p(_c(odom_T, np.float64).reshape(16)),
                     _p(_c(odom_cov, np.float64).reshape(36)), int(seed), int(step), _p(out), _p(delta))
    return out, delta


def init_uniform(n, lo, hi, seed):
    out = np.zeros((n, 7))
    lib().or_init_uniform(int(n), _p(_c(lo, np.float64)), _p(_c(hi, np.float64)), int(seed), _p(out))
    return out


# ---------------------------------------------------------------------------
# One filter step, in the paper's order.
# ---------------------------------------------------------------------------
@dataclass
class OracleFilter:
    map: OracleMap
    params: Params
    poses: np.ndarray                      # (n, 7) float32, the state
    ids: np.ndarray = None                 # (n, K) int32 lists, -1 padded
    logprior: np.ndarray = None            # (n,) float64
    step_index: int = 0
    nthreads: int = 0
    map_lo: np.ndarray = field(default=None)
    map_hi: np.ndarray = field(default=None)

    def __post_init__(self):
        n = len(self.poses)
        self.poses = _c(self.poses, np.float32).reshape(n, 7)
        if self.ids is None:
            self.ids = np.full((n, self.params.K), -1, np.int32)
            self.ids[:, 0] = np.arange(n, dtype=np.int32)
        if self.logprior is None:
            self.logprior = np.zeros(n)
        if self.map_lo is None:
            v = self.map.valid.astype(bool)
            self.map_lo = self.map.pts[v].min(0).astype(np.float64)
            self.map_hi = self.map.pts[v].max(0).astype(np.float64)

    def step(self, scan, odom_T=None, odom_cov=None):
        """One filter step on a scan (sensor frame, (n_s, 3)); returns every
        intermediate. An empty scan runs prediction, the neighbour update and
        the posterior smoothing with a zero log-likelihood (blackout step)."""
        P = self.params
        out = {}
        if odom_T is None:
            odom_T = np.eye(4)
        if odom_cov is None:
            odom_cov = np.zeros((6, 6))
        s = self.step_index
        # prediction (Sec. III-B, Eq. 1); with no motion and no noise it is the
        # identity and the stored FP32 poses are kept as they are
        if np.array_equal(np.asarray(odom_T, np.float64), np.eye(4)) and not np.any(odom_cov):
            pred = self.poses.astype(np.float64)
        else:
            pred, _ = predict(self.poses, odom_T, odom_cov, P.seed, s)
        poses = pred.astype(np.float32)
        out["pred_poses"] = pred
        out["poses_in"] = poses
        # scan Gaussians (Sec. III-C)
        scan = _c(scan, np.float32).reshape(-1, 3)
        if len(scan):
            sn, sv, _, _ = point_normals(scan, P.r_cov, P.cov_k, P.cov_min, nthreads=self.nthreads)
        else:
            sn, sv = np.zeros((0, 3)), np.zeros(0, np.uint8)
        out["scan_normals"], out["scan_valid"] = sn, sv
        # neighbour list update (Algorithm 1; Eq. 9, 10)
        q, t, d = lsh_draw(P.seed, s, self.map_lo, self.map_hi, P.lsh_sigma)
        out["lsh"] = (q, t, d)
        keys = lsh_keys(poses, q, t, d, P)
        out.update(keys=keys["keys"], buckets=keys["buckets"], lsh_flags=keys["flags"])
        srt = bucket_sort(keys["buckets"])
        out.update(srt)
        mg = neighbor_merge(poses, self.ids, srt, P, nthreads=self.nthreads)
        out.update(nbr_ids=mg["ids"], nbr_k=mg["k"], nbr_d=mg["d"], merge_flags=mg["flags"])
        n = len(poses)
        if len(scan) and sv.any():
            # likelihood evaluation (Eq. 2-4)
            lk = likelihood(self.map, poses, scan, sn, sv, P, nthreads=self.nthreads)
            out.update(H=lk["H"], b=lk["b"], loglik=lk["loglik"], n_in=lk["n_in"], amb=lk["amb"])
            # particle state update (Eq. 4-6)
            psi, ok = gn_solve(lk["H"], lk["b"], lk["n_in"], P)
            pinv = svgd_precond_matrices(lk["H"], ok, P) if P.svgd_precond else None
            phi, newp = svgd(poses, mg["ids"], mg["k"], mg["d"], psi, P, pinv)
            out.update(psi=psi, phi=phi, new_poses=newp)
            loglik = lk["loglik"]
        else:
            loglik = np.zeros(n)
            out.update(loglik=loglik, new_poses=poses.astype(np.float64))
        # posterior probability update (Eq. 11)
        p0, p, best = posterior(self.logprior, loglik, mg["ids"], mg["k"], P.post_iters, P.post_floor)
        out.update(post_init=p0, post=p, best=best)
        # the state is stored in FP32
        self.poses = out["new_poses"].astype(np.float32)
        self.ids = mg["ids"]
        with np.errstate(divide="ignore"):
            self.logprior = np.log(p)
        out["best_pose"] = self.poses[best].copy()
        self.step_index += 1
        return out
