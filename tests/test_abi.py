"""CPU checks of the boundary: the CUDA library builds for sm_103a, loads, and
exports every entry point the headers in include/ declare; parameter presets
agree with the oracle's readings. No kernel runs here."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "megaparticles.h")
HEADERS = [HEADER, os.path.join(ROOT, "include", "mp_proposal.h")]
PROBE_HEADER = os.path.join(ROOT, "include", "mp_probe.h")


def declared(headers=(HEADER,)):
    names = set()
    for h in headers:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(mp_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    from paper_2404_16370_gb300 import build as B
    return B.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("mp_init_map", "mp_init_particles", "mp_step", "mp_get_posterior", "mp_destroy", "mp_last_error"):
        assert must in names


def exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    return set(re.findall(r"\sT\s(mp_[a-z_0-9]+)$", out, flags=re.M))


def test_library_exports_every_declared_symbol(built):
    missing = [n for n in declared(HEADERS) if n not in exported(built)]
    assert not missing, missing


def test_probe_library_is_apart_from_the_filter_library(built):
    """The benchmark's measurement helpers (include/mp_probe.h) are exported by
    libmp_probe.so and not by libmp.so."""
    from paper_2404_16370_gb300 import build as B
    probe = declared((PROBE_HEADER,))
    assert set(probe) == {"mp_probe_random_reads", "mp_probe_fma_rate"}
    assert set(probe) <= exported(B.LIB_PROBE)
    assert not set(probe) & exported(built)


def test_library_loads_and_reports_without_gpu(built):
    from paper_2404_16370_gb300 import mp
    L = mp.lib()
    for n in declared():
        assert hasattr(L, n)
    # a call without a context records its message for mp_last_error(NULL)
    import ctypes as C
    ctx = C.c_void_p()
    assert L.mp_init_map(C.byref(ctx), None, 0, C.byref(mp.mp_default_params()), None) == mp.MP_EINVAL
    assert "mp_init_map: empty map or NULL argument" in mp.mp_last_error(None)
    L.mp_posterior_init_noalloc.argtypes = [C.c_void_p] * 2 + [C.c_int64] + [C.c_void_p] * 3
    assert L.mp_posterior_init_noalloc(None, None, 4, None, None, None) == mp.MP_EINVAL
    assert "NULL loglik" in mp.mp_last_error(None)
    p = mp.mp_default_params(mp.MP_PRESET_OUTDOOR, 1 << 20)
    assert p.n_buckets_log2 == 20 and p.K == 32 and abs(p.nnf_res - 0.2) < 1e-7
    with pytest.raises(mp.MPError):
        mp.mp_default_params(7, 10)


@pytest.mark.parametrize("preset,n", [(0, 4096), (1, 1 << 20), (0, 3), (1, 5000)])
def test_presets_match_oracle_readings(built, oracle, preset, n):
    from paper_2404_16370_gb300 import mp
    g = mp.mp_default_params(preset, n)
    o = oracle.Params.box_room(n) if preset == 0 else oracle.Params.outdoor(n)
    pairs = [("nnf_res", "res"), ("r_max", "r_max"), ("c_max", "c_max"), ("sigma_r", "sigma_r"),
             ("sigma_t", "sigma_t"), ("alpha", "alpha"), ("lsh_sigma", "lsh_sigma"), ("lambda_", "lam"),
             ("eps", "eps_damp"), ("eps_cov", "eps_cov"), ("r_cov", "r_cov"), ("K", "K"), ("C", "C"),
             ("cov_k", "cov_k"), ("cov_min", "cov_min"), ("post_iters", "post_iters"),
             ("n_buckets_log2", "nb_log2"), ("seed", "seed"), ("post_floor", "post_floor")]
    for gk, ok in pairs:
        assert abs(float(getattr(g, gk)) - float(getattr(o, ok))) <= 1e-7 * max(1.0, abs(float(getattr(o, ok)))), gk


def test_checked_build_exports_the_same_symbols(built):
    """The checked build (bounds-checked kernels, synchronised launches) is
    the same boundary: every declared entry point, plus nothing missing."""
    from paper_2404_16370_gb300 import build as B
    lib = B.build(checked=True)
    assert lib.endswith("libmp_checked.so")
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(mp_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in declared(HEADERS) if n not in exported]
    assert not missing, missing
    assert "mp_checked_sync" in out   # the host side of the checks is compiled in


def test_post_floor_is_validated_before_any_device_work(built):
    """mp_params.post_floor outside [0, 700] nats is refused by mp_init_map
    (parameters are checked before anything touches the device)."""
    import ctypes as C
    from paper_2404_16370_gb300 import mp
    L = mp.lib()
    pts = (C.c_float * 3)(0.0, 0.0, 0.0)
    for bad in (-1.0, 701.0, float("nan")):
        p = mp.mp_default_params(mp.MP_PRESET_BOX_ROOM, 64, post_floor=bad)
        ctx = C.c_void_p()
        assert L.mp_init_map(C.byref(ctx), pts, 1, C.byref(p), None) == mp.MP_EINVAL
        assert "post_floor" in mp.mp_last_error(None)
    assert mp.mp_default_params(mp.MP_PRESET_OUTDOOR, 64).post_floor == 700.0
