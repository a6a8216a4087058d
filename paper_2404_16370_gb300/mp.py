"""ctypes binding of libmp.so (include/megaparticles.h), one function per C
entry point with the same name. Argument marshalling only: every step of the
filter runs in the library's CUDA kernels. Arrays may be numpy arrays (host)
or torch tensors (host or CUDA; contiguous); outputs default to new numpy
arrays. Raises MPError on a non-zero return code, and ImportError when the
library has not been built (there is no CPU fallback)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MP_CHECKED=1: the checked build (bounds-checked kernels, every launch synchronised)
LIB_PATH = os.path.join(_HERE, {"1": "libmp_checked.so", "lite": "libmp_checked_lite.so"}.get(
    os.environ.get("MP_CHECKED", ""), "libmp.so"))

MP_OK, MP_EINVAL, MP_ENOMEM, MP_ECUDA, MP_ETIMEOUT, MP_ENOTINIT = 0, -1, -2, -3, -4, -5
MP_PRESET_BOX_ROOM, MP_PRESET_OUTDOOR = 0, 1

MP_STAGE_PREDICT = 0x001
MP_STAGE_SCAN = 0x002
MP_STAGE_LSH = 0x004
MP_STAGE_SORT = 0x008
MP_STAGE_MERGE = 0x010
MP_STAGE_LIKELIHOOD = 0x020
MP_STAGE_SOLVE = 0x040
MP_STAGE_SVGD = 0x080
MP_STAGE_POSTERIOR = 0x100
MP_STAGE_ALL = 0x1FF
STAGE_NAMES = ["predict", "scan", "lsh", "sort", "merge", "likelihood", "solve", "svgd", "posterior"]

MP_BUF_POSES, MP_BUF_LOG_PRIOR, MP_BUF_KEYS, MP_BUF_BUCKETS, MP_BUF_SORTED_IDS = 1, 2, 3, 4, 5
MP_BUF_SEGMENTS, MP_BUF_NBR_IDS, MP_BUF_NBR_K, MP_BUF_NBR_D, MP_BUF_GN = 6, 7, 8, 9, 10
MP_BUF_PSI, MP_BUF_POST, MP_BUF_POST_INIT, MP_BUF_LOGLIK, MP_BUF_SCAN_NORMALS = 11, 12, 13, 14, 15
MP_BUF_SCAN_VALID, MP_BUF_MAP_NORMALS, MP_BUF_MAP_VALID, MP_BUF_LSH, MP_BUF_PHI = 16, 17, 18, 19, 20
MP_BUF_VISIT_ORDER = 21

# element type and trailing shape of each buffer
_BUF = {
    MP_BUF_POSES: (np.float32, (7,)), MP_BUF_LOG_PRIOR: (np.float64, ()), MP_BUF_KEYS: (np.uint32, ()),
    MP_BUF_BUCKETS: (np.uint32, ()), MP_BUF_SORTED_IDS: (np.int32, ()), MP_BUF_SEGMENTS: (np.int32, (2,)),
    MP_BUF_NBR_IDS: (np.int32, ("K",)), MP_BUF_NBR_K: (np.float32, ("K",)), MP_BUF_NBR_D: (np.float32, ("K", 6)),
    MP_BUF_GN: (np.float32, (29,)), MP_BUF_PSI: (np.float32, (6,)), MP_BUF_POST: (np.float64, ()),
    MP_BUF_POST_INIT: (np.float64, ()), MP_BUF_LOGLIK: (np.float32, ()), MP_BUF_SCAN_NORMALS: (np.float32, (3,)),
    MP_BUF_SCAN_VALID: (np.uint8, ()), MP_BUF_MAP_NORMALS: (np.float32, (3,)), MP_BUF_MAP_VALID: (np.uint8, ()),
    MP_BUF_LSH: (np.float64, ()), MP_BUF_PHI: (np.float32, (6,)), MP_BUF_VISIT_ORDER: (np.int32, ()),
}


class mp_params(C.Structure):
    _fields_ = [("nnf_res", C.c_float), ("r_max", C.c_float), ("c_max", C.c_float),
                ("sigma_r", C.c_float), ("sigma_t", C.c_float), ("alpha", C.c_float), ("lsh_sigma", C.c_float),
                ("lambda_", C.c_float), ("eps", C.c_float), ("eps_cov", C.c_float), ("r_cov", C.c_float),
                ("K", C.c_int32), ("C", C.c_int32), ("cov_k", C.c_int32), ("cov_min", C.c_int32),
                ("post_iters", C.c_int32), ("n_buckets_log2", C.c_int32), ("max_scan", C.c_int32),
                ("seed", C.c_uint64), ("svgd_precond", C.c_int32), ("post_floor", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"megaparticles error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        V, P, I64, I32, U32, U64, D = C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
        L.mp_default_params.argtypes = [C.POINTER(mp_params), C.c_int, I64]
        L.mp_init_map.argtypes = [C.POINTER(V), P, I64, C.POINTER(mp_params), V]
        L.mp_init_map_shared.argtypes = [C.POINTER(V), V, C.POINTER(mp_params), V]
        L.mp_init_particles.argtypes = [V, I64, P, P, P, P]
        L.mp_step.argtypes = [V, P, I32, P, P]
        L.mp_get_posterior.argtypes = [V, P, P, P, P]
        L.mp_destroy.argtypes = [V]
        L.mp_last_error.argtypes = [V]
        L.mp_last_error.restype = C.c_char_p
        L.mp_set_scan.argtypes = [V, P, I32]
        L.mp_set_odometry.argtypes = [V, P, P]
        L.mp_run_stages.argtypes = [V, U32]
        L.mp_set_step_index.argtypes = [V, U64]
        L.mp_buffer_size.argtypes = [V, C.c_int, C.POINTER(I64)]
        L.mp_get_buffer.argtypes = [V, C.c_int, P, I64]
        L.mp_set_buffer.argtypes = [V, C.c_int, P, I64]
        L.mp_nnf_query.argtypes = [V, P, I64, P]
        L.mp_map_info.argtypes = [V, P, P, P, P, P]
        L.mp_set_timing.argtypes = [V, C.c_int]
        L.mp_stage_times.argtypes = [V, P, P, C.POINTER(I64)]
        L.mp_kernel_launches.argtypes = [V, C.POINTER(I64)]
        L.mp_set_precision.argtypes = [V, C.c_int]
        for f in ("mp_default_params", "mp_init_map", "mp_init_map_shared", "mp_init_particles", "mp_step", "mp_get_posterior", "mp_destroy",
                  "mp_set_scan", "mp_set_odometry", "mp_run_stages", "mp_set_step_index", "mp_buffer_size",
                  "mp_get_buffer", "mp_set_buffer", "mp_nnf_query", "mp_map_info", "mp_set_timing",
                  "mp_stage_times", "mp_kernel_launches", "mp_set_precision"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


_TORCH_NAME = {"float16": "torch.float16", "float32": "torch.float32", "float64": "torch.float64",
               "int32": "torch.int32", "uint32": "torch.uint32", "int64": "torch.int64", "uint8": "torch.uint8"}


def _ptr(x, dtype=None, shape=None, size=None, out=False):
    """(pointer, keep-alive) of None, a numpy array or a torch tensor.

    The library reads (or, out=True, writes) exactly the elements the caller
    describes, so mismatches are refused here, before the call: dtype is the
    element type the library uses (numpy inputs are converted to it; torch
    tensors and every output must already have it), shape the expected shape
    (-1 = any extent), size the expected element count. Outputs must be
    contiguous (a converted copy would not receive the result)."""
    if x is None:
        return None, None
    if shape is not None:
        got = tuple(int(d) for d in x.shape)
        if len(got) != len(shape) or any(w != -1 and w != d for w, d in zip(shape, got)):
            raise ValueError(f"array of shape {got}: the library expects {tuple(shape)} (-1: any extent)")
    if size is not None:
        n = int(x.numel()) if hasattr(x, "numel") else int(np.size(x))
        if n != size:
            raise ValueError(f"array of {n} elements: the library expects {size}")
    if hasattr(x, "data_ptr"):               # torch tensor
        if dtype is not None and str(x.dtype) != _TORCH_NAME.get(np.dtype(dtype).name):
            raise TypeError(f"tensor of {x.dtype}: the library uses {np.dtype(dtype).name}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr()), x
    if out:
        if not isinstance(x, np.ndarray) or (dtype is not None and x.dtype != np.dtype(dtype)) \
                or not x.flags.c_contiguous or not x.flags.writeable:
            raise TypeError(f"output must be a writeable C-contiguous {np.dtype(dtype).name} array")
        return x.ctypes.data_as(C.c_void_p), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), a


def _check(rc, ctx):
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(ctx))


def mp_last_error(ctx) -> str:
    return lib().mp_last_error(ctx).decode(errors="replace")


def mp_default_params(preset=MP_PRESET_BOX_ROOM, n_particles=4096, **overrides) -> mp_params:
    p = mp_params()
    rc = lib().mp_default_params(C.byref(p), int(preset), int(n_particles))
    if rc != MP_OK:
        raise MPError(rc, f"unknown preset {preset}")
    for k, v in overrides.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


def mp_init_map(xyz, params: mp_params, cuda_stream=None):
    ctx = C.c_void_p()
    ptr, keep = _ptr(xyz, np.float32, shape=(-1, 3))
    n = int(xyz.shape[0])
    rc = lib().mp_init_map(C.byref(ctx), ptr, n, C.byref(params), C.c_void_p(cuda_stream) if cuda_stream else None)
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))
    return ctx


def mp_init_map_shared(src, params: mp_params, cuda_stream=None):
    """A context on src's device map (no copy; freed with the last context on it)."""
    ctx = C.c_void_p()
    rc = lib().mp_init_map_shared(C.byref(ctx), src, C.byref(params), C.c_void_p(cuda_stream) if cuda_stream else None)
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))
    return ctx


def mp_init_particles(ctx, n_particles, lo=None, hi=None, poses=None, log_prior=None):
    pl, kl = _ptr(lo, np.float32, size=6)
    ph, kh = _ptr(hi, np.float32, size=6)
    n = int(n_particles)   # n <= 0 is the library's to refuse (MP_EINVAL)
    pp, kp = _ptr(poses, np.float32, shape=(n, 7) if n > 0 else None)
    pr, kr = _ptr(log_prior, np.float64, size=n if n > 0 else None)
    _check(lib().mp_init_particles(ctx, int(n_particles), pl, ph, pp, pr), ctx)


def mp_step(ctx, scan, odom_T=None, odom_cov=None):
    ps, ks = _ptr(scan, np.float32, shape=(-1, 3))
    pt, kt = _ptr(odom_T, np.float64, size=16)
    pc, kc = _ptr(odom_cov, np.float64, size=36)
    n = 0 if scan is None else int(scan.shape[0])
    _check(lib().mp_step(ctx, ps, n, pt, pc), ctx)


def mp_get_posterior(ctx, poses_out=None, prob_out=None):
    best = np.zeros(7, np.float32)
    bp = np.zeros(1, np.float64)
    if poses_out is not None or prob_out is not None:
        n = mp_buffer_size(ctx, MP_BUF_LOG_PRIOR)
    po, ko = _ptr(poses_out, np.float32, size=None if poses_out is None else 7 * n, out=True)
    pr, kr = _ptr(prob_out, np.float64, size=None if prob_out is None else n, out=True)
    _check(lib().mp_get_posterior(ctx, po, pr, best.ctypes.data_as(C.c_void_p), bp.ctypes.data_as(C.c_void_p)), ctx)
    return best, float(bp[0])


def mp_destroy(ctx):
    if ctx:
        lib().mp_destroy(ctx)


def mp_set_scan(ctx, scan):
    ps, ks = _ptr(scan, np.float32, shape=(-1, 3))
    _check(lib().mp_set_scan(ctx, ps, 0 if scan is None else int(scan.shape[0])), ctx)


def mp_set_odometry(ctx, odom_T=None, odom_cov=None):
    pt, kt = _ptr(odom_T, np.float64, size=16)
    pc, kc = _ptr(odom_cov, np.float64, size=36)
    _check(lib().mp_set_odometry(ctx, pt, pc), ctx)


def mp_run_stages(ctx, mask):
    _check(lib().mp_run_stages(ctx, int(mask)), ctx)


def mp_set_step_index(ctx, step):
    _check(lib().mp_set_step_index(ctx, int(step)), ctx)


def mp_buffer_size(ctx, which) -> int:
    n = C.c_int64()
    _check(lib().mp_buffer_size(ctx, int(which), C.byref(n)), ctx)
    return int(n.value)


def _shape(which, count, K):
    dt, tail = _BUF[which]
    tail = tuple(K if t == "K" else t for t in tail)
    per = int(np.prod(tail)) if tail else 1
    return dt, (count // per,) + tail


def mp_get_buffer(ctx, which, K=None, out=None):
    """Copy a library buffer into a new numpy array, or into `out` (numpy or
    torch, host or device); the element count passed is out's own, so the
    library rejects an `out` of the wrong size."""
    if out is None:
        count = mp_buffer_size(ctx, which)
        dt, shape = _shape(which, count, K if K is not None else _guess_k(ctx, which, count))
        out = np.empty(shape, dt)
    else:
        count = int(out.numel()) if hasattr(out, "numel") else int(out.size)
    po, ko = _ptr(out, _BUF[which][0], out=True)
    _check(lib().mp_get_buffer(ctx, int(which), po, count), ctx)
    return out


def _guess_k(ctx, which, count):
    if _BUF[which][1] and _BUF[which][1][0] == "K":
        n = mp_buffer_size(ctx, MP_BUF_LOG_PRIOR)
        per = count // max(n, 1)
        return per // 6 if which == MP_BUF_NBR_D else per
    return None


def mp_set_buffer(ctx, which, src):
    dt, _ = _BUF[which]
    ps, ks = _ptr(src, dt)
    count = int(np.prod(src.shape))
    _check(lib().mp_set_buffer(ctx, int(which), ps, count), ctx)


def mp_nnf_query(ctx, vox):
    v = np.ascontiguousarray(vox, np.int32).reshape(-1, 3)
    out = np.empty(len(v), np.int32)
    _check(lib().mp_nnf_query(ctx, v.ctypes.data_as(C.c_void_p), len(v), out.ctypes.data_as(C.c_void_p)), ctx)
    return out


def mp_map_info(ctx):
    o = np.zeros(3, np.float32); d = np.zeros(3, np.int32); inv = np.zeros(1, np.float32)
    off = np.zeros(3, np.float32); nv = np.zeros(1, np.int64)
    _check(lib().mp_map_info(ctx, *(a.ctypes.data_as(C.c_void_p) for a in (o, d, inv, off, nv))), ctx)
    return dict(origin=o, dims=d, inv_res=float(inv[0]), off=off, n_valid=int(nv[0]))


def mp_set_timing(ctx, enable=True):
    _check(lib().mp_set_timing(ctx, int(bool(enable))), ctx)


def mp_stage_times(ctx):
    """(per-stage total ms, per-stage run counts, likelihood pairs) since timing was enabled."""
    ms = np.zeros(9, np.float32)
    runs = np.zeros(9, np.int64)
    pairs = C.c_int64()
    _check(lib().mp_stage_times(ctx, ms.ctypes.data_as(C.c_void_p), runs.ctypes.data_as(C.c_void_p),
                                C.byref(pairs)), ctx)
    return dict(zip(STAGE_NAMES, ms.tolist())), dict(zip(STAGE_NAMES, runs.tolist())), int(pairs.value)


MP_DEBUG_WAIT_BUDGET, MP_DEBUG_STARVE_TX, MP_DEBUG_STARVE_BARRIER = 1, 2, 3


def mp_debug_set(ctx, what, value):
    L = lib()
    L.mp_debug_set.argtypes = [C.c_void_p, C.c_int, C.c_int64]
    L.mp_debug_set.restype = C.c_int
    _check(L.mp_debug_set(ctx, int(what), int(value)), ctx)


def _device_tensor(x, name):
    """x as a torch tensor on the current CUDA device, else TypeError: the
    allocation-free entry point dereferences its pointers as device memory of
    the current device (the library refuses anything else too)."""
    if not (hasattr(x, "data_ptr") and hasattr(x, "is_cuda")):
        raise TypeError(f"{name}: expected a CUDA tensor, got {type(x).__name__}")
    if not x.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor, got one on {x.device}")
    import torch
    if x.device.index != torch.cuda.current_device():
        raise TypeError(f"{name}: tensor on {x.device}, the current device is cuda:{torch.cuda.current_device()}")
    return x


def mp_posterior_init_noalloc(log_prior, loglik, post_out, best_out, cuda_stream=None):
    """Device tensors of the current device in, device tensors out; allocates
    nothing (see the C header). log_prior may be None (uniform prior)."""
    L = lib()
    if not getattr(L, "_noalloc_declared", False):
        L.mp_posterior_init_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                                C.c_void_p]
        L.mp_posterior_init_noalloc.restype = C.c_int
        L._noalloc_declared = True
    for x, name in ((log_prior, "log_prior"), (loglik, "loglik"), (post_out, "post_out"), (best_out, "best_out")):
        if x is not None or name != "log_prior":
            _device_tensor(x, name)
    n = int(loglik.shape[0])
    lp, klp = _ptr(log_prior, np.float64, size=n)
    ll, kll = _ptr(loglik, np.float32, size=n)
    po, kpo = _ptr(post_out, np.float64, size=n, out=True)
    bo, kbo = _ptr(best_out, np.int64, size=1, out=True)
    rc = L.mp_posterior_init_noalloc(lp, ll, n, po, bo, C.c_void_p(cuda_stream) if cuda_stream else None)
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))


def mp_kernel_launches(ctx) -> int:
    n = C.c_int64()
    _check(lib().mp_kernel_launches(ctx, C.byref(n)), ctx)
    return int(n.value)


MP_PREC_FP32, MP_PREC_BF16, MP_PREC_FP16 = 0, 1, 2


def mp_set_precision(ctx, precision):
    """Arithmetic precision of the likelihood stage: MP_PREC_FP32 (default),
    MP_PREC_BF16 or MP_PREC_FP16 (16-bit per-pair arithmetic, FP32 sums)."""
    _check(lib().mp_set_precision(ctx, int(precision)), ctx)


# ---------------------------------------------------------------------------
# learned proposal (include/mp_proposal.h): device tensors in and out
MP_PN_OUT, MP_PN_COMPONENTS = 416, 32


def _pn_lib():
    L = lib()
    if not getattr(L, "_pn_declared", False):
        V, P, I64, U64 = C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64
        L.mp_pn_sim_box_room.argtypes = [P, C.c_int, C.c_float, C.c_float, P, I64, P, C.c_int, C.c_float, U64, P, V]
        L.mp_pn_create.argtypes = [C.POINTER(V), C.c_int, C.c_int, C.c_float, P, P, U64, V]
        L.mp_pn_destroy.argtypes = [V]
        L.mp_pn_num_params.argtypes = [V, C.POINTER(I64)]
        L.mp_pn_get_params.argtypes = [V, P]
        L.mp_pn_set_params.argtypes = [V, P]
        L.mp_pn_forward.argtypes = [V, P, C.c_int, P]
        L.mp_pn_loss_grad.argtypes = [V, P, P, C.c_int, P, P]
        L.mp_pn_adam_step.argtypes = [V, C.c_float, C.c_float, C.c_float, C.c_float]
        L.mp_pn_sample.argtypes = [V, P, I64, U64, P]
        L.mp_pn_set_precision.argtypes = [V, C.c_int]
        L.mp_pn_status.argtypes = [V]
        for f in ("mp_pn_sim_box_room", "mp_pn_create", "mp_pn_destroy", "mp_pn_num_params", "mp_pn_get_params",
                  "mp_pn_set_params", "mp_pn_forward", "mp_pn_loss_grad", "mp_pn_adam_step", "mp_pn_sample",
                  "mp_pn_set_precision", "mp_pn_status"):
            getattr(L, f).restype = C.c_int
        L._pn_declared = True
    return L


def _pn_check(rc, what):
    if rc != MP_OK:
        raise MPError(rc, f"{what} failed: {mp_last_error(None)}")


def _dev(t, shape=None, numel=None):
    """data_ptr of a contiguous CUDA float32 tensor; shape (-1: any extent)
    or numel, when given, is what the library reads or writes there."""
    if not hasattr(t, "data_ptr"):
        raise ValueError("expected a CUDA tensor")
    if str(t.dtype) != "torch.float32":
        raise TypeError(f"tensor of {t.dtype}: the library uses float32")
    if shape is not None:
        got = tuple(int(d) for d in t.shape)
        if len(got) != len(shape) or any(w != -1 and w != d for w, d in zip(shape, got)):
            raise ValueError(f"tensor of shape {got}: the library expects {tuple(shape)} (-1: any extent)")
    if numel is not None and int(t.numel()) != numel:
        raise ValueError(f"tensor of {int(t.numel())} elements: the library expects {numel}")
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


_pn_points = {}   # network pointer -> points per scan


def _pn_scan_shape(net):
    return (-1, _pn_points.get(net.value if isinstance(net, C.c_void_p) else net, -1), 3)


def mp_pn_sim_box_room(boxes, half, height, poses, dirs, noise, seed, out, cuda_stream=None):
    """Ray-cast B x P box-room scans into out (B, P, 3); all tensors on the GPU."""
    B, P = int(poses.shape[0]), int(dirs.shape[0])
    pb, pp, pd = _dev(boxes, (-1, 7)), _dev(poses, (B, 7)), _dev(dirs, (P, 3))
    po = _dev(out, (B, P, 3))
    _pn_check(_pn_lib().mp_pn_sim_box_room(pb, int(boxes.shape[0]), float(half), float(height), pp,
                                           B, pd, P, float(noise),
                                           int(seed) & (2 ** 64 - 1), po,
                                           C.c_void_p(cuda_stream) if cuda_stream else None), "mp_pn_sim_box_room")


def mp_pn_create(n_points, max_batch, in_scale, scale, offset, seed=0, cuda_stream=None):
    net = C.c_void_p()
    sc = np.ascontiguousarray(scale, np.float32)
    of = np.ascontiguousarray(offset, np.float32)
    _pn_check(_pn_lib().mp_pn_create(C.byref(net), int(n_points), int(max_batch), float(in_scale),
                                     sc.ctypes.data_as(C.c_void_p), of.ctypes.data_as(C.c_void_p),
                                     int(seed) & (2 ** 64 - 1), C.c_void_p(cuda_stream) if cuda_stream else None),
              "mp_pn_create")
    _pn_points[net.value] = int(n_points)
    return net


def mp_pn_destroy(net):
    _pn_points.pop(net.value if isinstance(net, C.c_void_p) else net, None)
    _pn_check(_pn_lib().mp_pn_destroy(net), "mp_pn_destroy")


def mp_pn_num_params(net) -> int:
    n = C.c_int64()
    _pn_check(_pn_lib().mp_pn_num_params(net, C.byref(n)), "mp_pn_num_params")
    return int(n.value)


def mp_pn_get_params(net, out):
    po = _dev(out, numel=mp_pn_num_params(net))
    _pn_check(_pn_lib().mp_pn_get_params(net, po), "mp_pn_get_params")


def mp_pn_set_params(net, params):
    pp = _dev(params, numel=mp_pn_num_params(net))
    _pn_check(_pn_lib().mp_pn_set_params(net, pp), "mp_pn_set_params")


def mp_pn_forward(net, scans, out):
    B = int(scans.shape[0])
    ps, po = _dev(scans, _pn_scan_shape(net)), _dev(out, (B, MP_PN_OUT))
    _pn_check(_pn_lib().mp_pn_forward(net, ps, B, po), "mp_pn_forward")


def mp_pn_loss_grad(net, scans, targets, loss, grad=None):
    B = int(scans.shape[0])
    ps, pt, pl = _dev(scans, _pn_scan_shape(net)), _dev(targets, (B, 6)), _dev(loss, numel=1)
    pg = _dev(grad, numel=mp_pn_num_params(net)) if grad is not None else None
    _pn_check(_pn_lib().mp_pn_loss_grad(net, ps, pt, B, pl, pg), "mp_pn_loss_grad")


def mp_pn_adam_step(net, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _pn_check(_pn_lib().mp_pn_adam_step(net, float(lr), float(beta1), float(beta2), float(eps)), "mp_pn_adam_step")


def mp_pn_set_precision(net, precision):
    """MP_PREC_BF16: the per-point layers on the tensor cores (the default for
    scans of a multiple of 128 points); MP_PREC_FP32: on the CUDA cores."""
    _pn_check(_pn_lib().mp_pn_set_precision(net, int(precision)), "mp_pn_set_precision")


def mp_pn_status(net):
    """Waits for the network's stream; raises MPError (MP_ETIMEOUT) if a
    bounded wait of the tensor-core forward pass gave up."""
    _pn_check(_pn_lib().mp_pn_status(net), "mp_pn_status")


def mp_pn_sample(net, mix, n, seed, out):
    pm, po = _dev(mix, numel=MP_PN_OUT), _dev(out, (int(n), 7))
    _pn_check(_pn_lib().mp_pn_sample(net, pm, int(n), int(seed) & (2 ** 64 - 1), po), "mp_pn_sample")


# ---------------------------------------------------------------------------
# batched instances and the likelihood split


def mp_set_likelihood_split(ctx, split):
    L = lib()
    L.mp_set_likelihood_split.argtypes = [C.c_void_p, C.c_int]
    L.mp_set_likelihood_split.restype = C.c_int
    _check(L.mp_set_likelihood_split(ctx, int(split)), ctx)


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_declared", False):
        V = C.c_void_p
        L.mp_batch_create.argtypes = [C.POINTER(V), C.POINTER(V), C.c_int, V, C.POINTER(V), V]
        L.mp_batch_step.argtypes = [V, C.POINTER(V), V, V]
        L.mp_batch_split.argtypes = [V, C.c_int, C.POINTER(C.c_int)]
        L.mp_batch_destroy.argtypes = [V]
        for f in ("mp_batch_create", "mp_batch_step", "mp_batch_split", "mp_batch_destroy"):
            getattr(L, f).restype = C.c_int
        L._batch_declared = True
    return L


def mp_batch_create(ctxs, n_scan, cuda_stream, tune_scans=None):
    """ctxs: contexts (their streams may be cuda_stream itself); n_scan: fixed scan size of each;
    tune_scans: list of (n_scan[i], 3) float32 arrays or None."""
    n = len(ctxs)
    arr = (C.c_void_p * n)(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    ns = np.ascontiguousarray(n_scan, np.int32)
    if ns.shape != (n,):
        raise ValueError(f"n_scan holds {ns.size} sizes for {n} contexts")
    keep = []
    tp = None
    if tune_scans is not None:
        if len(tune_scans) != n:
            raise ValueError(f"{len(tune_scans)} tuning scans for {n} contexts")
        ptrs = []
        for i, sc in enumerate(tune_scans):
            a = _batch_scan(sc, int(ns[i]), i)
            keep.append(a)
            ptrs.append(a.ctypes.data)
        tp = (C.c_void_p * n)(*ptrs)
    b = C.c_void_p()
    rc = _batch_lib().mp_batch_create(C.byref(b), arr, n, ns.ctypes.data_as(C.c_void_p), tp,
                                      C.c_void_p(cuda_stream))
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))
    _batch_nscan[b.value] = [int(v) for v in ns]
    return b


def _batch_scan(sc, n_scan, i):
    """Instance i's host scan as the (n_scan, 3) float32 array the library copies from."""
    if hasattr(sc, "data_ptr"):
        raise TypeError("batched scans are host arrays (numpy)")
    a = np.ascontiguousarray(sc, np.float32)
    if a.shape != (n_scan, 3):
        raise ValueError(f"instance {i}: scan of shape {a.shape}, the batch was created for ({n_scan}, 3)")
    return a


_batch_nscan = {}   # batch pointer -> each instance's fixed scan size


def mp_batch_step(batch, scans, odom_T=None, odom_cov=None):
    n = len(scans)
    sizes = _batch_nscan.get(batch.value if isinstance(batch, C.c_void_p) else batch)
    if sizes is None:
        raise ValueError("not a live batch of this module")
    if n != len(sizes):
        raise ValueError(f"{n} scans for a batch of {len(sizes)} instances")
    keep = [_batch_scan(sc, sizes[i], i) for i, sc in enumerate(scans)]
    ptrs = (C.c_void_p * n)(*[a.ctypes.data for a in keep])
    T = None if odom_T is None else np.ascontiguousarray(odom_T, np.float64).reshape(n, 16)
    Q = None if odom_cov is None else np.ascontiguousarray(odom_cov, np.float64).reshape(n, 36)
    rc = _batch_lib().mp_batch_step(batch, ptrs, None if T is None else T.ctypes.data_as(C.c_void_p),
                                    None if Q is None else Q.ctypes.data_as(C.c_void_p))
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))


def mp_batch_split(batch, i) -> int:
    s = C.c_int()
    rc = _batch_lib().mp_batch_split(batch, int(i), C.byref(s))
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))
    return int(s.value)


def mp_batch_destroy(batch):
    _batch_nscan.pop(batch.value if isinstance(batch, C.c_void_p) else batch, None)
    rc = _batch_lib().mp_batch_destroy(batch)
    if rc != MP_OK:
        raise MPError(rc, mp_last_error(None))


def mp_stream_create() -> int:
    """A new non-blocking CUDA stream (its cudaStream_t as an int)."""
    L = lib()
    L.mp_stream_create.argtypes = [C.POINTER(C.c_void_p)]
    L.mp_stream_create.restype = C.c_int
    s = C.c_void_p()
    rc = L.mp_stream_create(C.byref(s))
    if rc != MP_OK:
        raise MPError(rc, "mp_stream_create failed")
    return int(s.value)


def mp_stream_destroy(stream):
    L = lib()
    L.mp_stream_destroy.argtypes = [C.c_void_p]
    L.mp_stream_destroy.restype = C.c_int
    rc = L.mp_stream_destroy(C.c_void_p(stream))
    if rc != MP_OK:
        raise MPError(rc, "mp_stream_destroy failed")


# ---------------------------------------------------------------------------
# scan-to-scan GICP odometry


def mp_gicp(ctx, src, tgt, init_T=None, max_iters=30):
    """DeltaT (4x4) mapping src (current scan) into tgt's frame (previous scan),
    Sigma^DeltaT = H^-1 (6x6), correspondences and iterations."""
    L = lib()
    L.mp_gicp.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                          C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    L.mp_gicp.restype = C.c_int
    sp, ks = _ptr(src, np.float32, shape=(-1, 3))
    tp, kt = _ptr(tgt, np.float32, shape=(-1, 3))
    if init_T is not None and np.size(init_T) != 16:
        raise ValueError("init_T must hold 16 values (row-major 4x4)")
    T0 = None if init_T is None else np.ascontiguousarray(init_T, np.float64)
    T = np.zeros(16)
    cov = np.zeros(36)
    nc, it = C.c_int32(), C.c_int32()
    _check(L.mp_gicp(ctx, sp, int(src.shape[0]), tp, int(tgt.shape[0]),
                     None if T0 is None else T0.ctypes.data_as(C.c_void_p), int(max_iters),
                     T.ctypes.data_as(C.c_void_p), cov.ctypes.data_as(C.c_void_p), C.byref(nc), C.byref(it)), ctx)
    return dict(T=T.reshape(4, 4), cov=cov.reshape(6, 6), n_corr=int(nc.value), iters=int(it.value))


def mp_step_gicp(ctx, scan, cov_scale=1.0):
    """mp_step with GICP odometry against the previous scan given here."""
    L = lib()
    L.mp_step_gicp.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_double]
    L.mp_step_gicp.restype = C.c_int
    if scan is None or len(scan) == 0:
        _check(L.mp_step_gicp(ctx, None, 0, float(cov_scale)), ctx)
        return
    sp, keep = _ptr(scan, np.float32, shape=(-1, 3))
    _check(L.mp_step_gicp(ctx, sp, int(scan.shape[0]), float(cov_scale)), ctx)


# ---------------------------------------------------------------------------
# measurement helpers of the benchmark (include/mp_probe.h, libmp_probe.so)

PROBE_PATH = os.path.join(_HERE, "libmp_probe.so")
_probe = None


def probe_lib():
    global _probe
    if _probe is None:
        if not os.path.exists(PROBE_PATH):
            raise ImportError(f"{PROBE_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(PROBE_PATH)
        L.mp_probe_random_reads.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                            C.POINTER(C.c_float), C.POINTER(C.c_int64)]
        L.mp_probe_fma_rate.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_float),
                                        C.POINTER(C.c_double)]
        for f in ("mp_probe_random_reads", "mp_probe_fma_rate"):
            getattr(L, f).restype = C.c_int
        _probe = L
    return _probe


def mp_probe_random_reads(words, blocks, reads_per_thread, repeats=5, cuda_stream=None):
    """(mean ms of one run, reads per run) of independent random 4-byte reads
    over `words` (a uint32/int32 tensor on the current CUDA device)."""
    _device_tensor(words, "words")
    ms, n = C.c_float(), C.c_int64()
    rc = probe_lib().mp_probe_random_reads(C.c_void_p(words.data_ptr()), int(words.numel()), int(blocks),
                                           int(reads_per_thread), int(repeats),
                                           C.c_void_p(cuda_stream) if cuda_stream else None, C.byref(ms), C.byref(n))
    if rc != MP_OK:
        raise MPError(rc, "mp_probe_random_reads: invalid argument or CUDA failure")
    return float(ms.value), int(n.value)


MP_FMA_FP32, MP_FMA_FP32X2, MP_FMA_FP64 = 0, 1, 2


def mp_probe_fma_rate(kind, blocks, iters, repeats=3, cuda_stream=None):
    """(mean ms of one run, flops of one run) of the FMA throughput probe."""
    ms, fl = C.c_float(), C.c_double()
    rc = probe_lib().mp_probe_fma_rate(int(kind), int(blocks), int(iters), int(repeats),
                                       C.c_void_p(cuda_stream) if cuda_stream else None, C.byref(ms), C.byref(fl))
    if rc != MP_OK:
        raise MPError(rc, "mp_probe_fma_rate: invalid argument or CUDA failure")
    return float(ms.value), float(fl.value)
