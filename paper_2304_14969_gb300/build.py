"""Builds libqsim.so from csrc/ with nvcc for sm_103a (GB300) only.

Each translation unit compiles in its own nvcc process (in parallel); the
objects are linked into ``paper_2304_14969_gb300/libqsim.so`` against the
shared CUDA runtime, so the process shares one runtime with PyTorch.
Usage: ``python -m paper_2304_14969_gb300.build [--verbose-ptxas]``.
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
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqsim.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqsim.so")


def sources() -> list:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _deps_mtime() -> float:
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files.append(os.path.join(ROOT, "include", "qsim.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, ptxas_verbose: bool) -> tuple:
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if ptxas_verbose and src.endswith(".cu"):
        cmd[1:1] = ["-Xptxas", "-v"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, p.returncode, p.stdout + p.stderr


def build(force: bool = False, ptxas_verbose: bool = False, quiet: bool = True) -> str:
    """Compiles (if stale) and returns the path of libqsim.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime() and not ptxas_verbose:
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sources()
    objs, logs = [], []
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        for src, obj, rc, log in ex.map(lambda s: _compile(s, ptxas_verbose), srcs):
            logs.append((src, log))
            if rc != 0:
                raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{log}")
            objs.append(obj)
    tmp = LIB + f".tmp{os.getpid()}"
    p = subprocess.run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs],
                       capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    os.replace(tmp, LIB)
    if not quiet or ptxas_verbose:
        for src, log in logs:
            if log.strip():
                print(f"== {os.path.basename(src)}\n{log}")
    return LIB


if __name__ == "__main__":
    build(force=True, ptxas_verbose="--verbose-ptxas" in sys.argv, quiet=False)
    print(LIB)
