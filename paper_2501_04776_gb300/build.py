"""Build the CUDA library libiqp_gb300.so in-tree (nvcc, sm_103a only).

Each translation unit compiles in parallel to an object file under _build/,
then nvcc links the shared library next to this file. The CUDA runtime is
linked statically and the driver API is reached through
cudaGetDriverEntryPointByVersion, so the library loads on machines without a
GPU driver (its symbols can be checked there) and only needs one at call time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "iqp")
LIB = os.path.join(HERE, "libiqp_gb300.so")
CHECKED_LIB = os.path.join(HERE, "libiqp_gb300_checked.so")
SOURCES = ["parity.cu", "simt.cu", "tc.cu", "bitflip.cu", "sparse.cu", "variants.cu", "loworder.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libiqp_gb300.so")
    return path


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(INCLUDE, "iqp.h")] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checks: bool = False) -> str:
    """Compile (what changed) and link the library. checks=True builds the
    self-checked variant (-DIQP_CHECKS: every kernel index derived from the
    caller's shapes is compared with its buffer's extent) into
    libiqp_gb300_checked.so beside the default library, from its own objects."""
    build_dir = BUILD + ("_checked" if checks else "")
    lib = CHECKED_LIB if checks else LIB
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    extra = list(extra or []) + (["-DIQP_CHECKS"] if checks else [])

    def compile_one(name: str) -> str:
        src = os.path.join(CSRC, name)
        obj = os.path.join(build_dir, name + ".o")
        if force or (extra and not checks) or _stale(obj, src):
            cmd = [cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {name}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or (extra and not checks) or not os.path.exists(lib) or any(
            os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + ".tmp"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":  # pragma: no cover
    args = sys.argv[1:]
    print(build(force="--force" in args, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas-v" in args else None))
