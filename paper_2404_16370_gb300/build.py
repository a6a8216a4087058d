"""Builds libmp.so (the CUDA library behind include/megaparticles.h) in-tree
for sm_103a: one nvcc job per translation unit, in parallel, then a shared
link. Host code is compiled without floating-point contraction (the NNF
geometry is an FP32 decision sequence). The benchmark's measurement helpers
(include/mp_probe.h, csrc/probe/) become a library of their own,
libmp_probe.so, built by the same call.

build(checked=True) (or `python -m paper_2404_16370_gb300.build --checked`)
makes libmp_checked.so with -DMP_CHECKED instead: kernels bound-check the
indices they read from data and every launch is synchronised, so that a fault
is reported at the kernel that caused it. mp.py loads it when MP_CHECKED=1 is
set in the environment. It is a debugging aid, several times slower."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmp.so")
LIB_CHECKED = os.path.join(HERE, "libmp_checked.so")
LIB_PROBE = os.path.join(HERE, "libmp_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", os.path.join(os.path.dirname(HERE), "include")]
# The filter-step kernels are built without implicit multiply-add contraction:
# each kernel body is instantiated twice (a context's own launch and the
# batch's grouped launch), and only explicit fma / __f*_rn operations round the
# same way in both whatever the surrounding code. The likelihood's arithmetic
# is explicit (packed f32x2 intrinsics, fmaf) and keeps the default flags.
NO_FMAD = {"k_update.cu", "k_neighbors.cu", "k_map.cu", "k_posterior.cu"}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked=False) -> str:
    """checked: False, True (printed checks) or "lite" (checks recorded by one
    atomic, no printf; libmp_checked_lite.so). The normal build also makes
    libmp_probe.so."""
    suffix = "_checked_lite" if checked == "lite" else "_checked" if checked else ""
    lib = _build_lib(CSRC, BUILD + suffix, os.path.join(HERE, f"libmp{suffix}.so"), force, verbose, ptxas_info,
                     checked)
    if not checked:
        _build_lib(os.path.join(CSRC, "probe"), BUILD + "_probe", LIB_PROBE, force, verbose, ptxas_info, False)
    return lib


def _build_lib(csrc, build_dir, lib, force, verbose, ptxas_info, checked) -> str:
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")))
    headers = sorted(glob.glob(os.path.join(csrc, "*.cuh"))) + sorted(
        glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")))
    objs = [os.path.join(build_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DMP_CHECKED"] if checked else []) + \
        (["-DMP_CHECKED_LITE"] if checked == "lite" else [])

    def compile_one(src_obj):
        src, obj = src_obj
        if not force and not ptxas_info and not _stale(obj, [src] + headers):
            return ""
        fmad = ["-fmad=false"] if os.path.basename(src) in NO_FMAD else []
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *fmad, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose or ptxas_info:
        for lg in logs:
            if lg:
                sys.stderr.write(lg)
    if force or ptxas_info or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="lite" if "--checked-lite" in sys.argv else "--checked" in sys.argv))
