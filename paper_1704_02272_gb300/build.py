"""Builds libpfac.so (host builder + sm_103a kernels) in-tree with nvcc.

Every translation unit is compiled in parallel for ``sm_103a`` only, then
linked into ``paper_1704_02272_gb300/_build/libpfac.so``.  Run as
``python paper_1704_02272_gb300/build.py`` (no import of the package, which
needs the built library) or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpfac.so")
CHECKED_LIB = os.path.join(BUILD, "libpfac_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
          "--expt-relaxed-constexpr"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpfac")
    return p


def sources():
    srcs = ["builder.cpp", "tune.cpp", "serve.cpp", "host.cpp", "match.cu", "noalloc.cu",
            "verify.cu", "resolve.cu", "scan_dense.cu", "table_io.cpp"] + [f"scan_bps{i}.cu" for i in range(1, 9)] + \
        [f"scan_r{b}_{g}.cu" for b in (8, 2) for g in ("g0_f", "g0_fe", "g1_f", "g1_fe", "d0", "d1")]
    return [os.path.join(CSRC, s) for s in srcs]


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(os.path.dirname(HERE), "include", "pfac.h")]


def _stale(obj, src, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    """Builds libpfac.so; with checked=True the bounds-checked library
    (PFAC_CHECKED: every table, shared-memory, queue and input index of the
    compressed-layout kernels range-checked) as libpfac_checked.so."""
    bdir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = CHECKED_LIB if checked else LIB
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    deps = headers()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, src, deps):
            cmd = [cc, *COMMON, *ARCH, *(["-DPFAC_CHECKED"] if checked else []), "-c", src, "-o", obj]
            if ptxas_info and src.endswith(".cu"):
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    if jobs:
        workers = min(len(jobs), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(workers) as ex:
            futs = [ex.submit(subprocess.run, c, capture_output=True, text=True) for c in jobs]
            for c, f in zip(jobs, futs):
                r = f.result()
                if verbose or ptxas_info:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed:\n" + " ".join(c) + "\n" + r.stdout + r.stderr)
    stale_lib = not os.path.exists(lib) or any(
        os.path.getmtime(o) > os.path.getmtime(lib) for o in objs)
    if force or jobs or stale_lib:
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([cc, "-shared", *ARCH, "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
