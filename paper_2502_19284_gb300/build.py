"""Build libspmv.so (sm_103a) in-tree with nvcc: one object per translation unit,
compiled in parallel, then linked into paper_2502_19284_gb300/_build/libspmv.so."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libspmv.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

UNITS = ["primitives", "convert", "spmv", "stage", "mergeb", "store", "cg", "pagerank", "batch", "serve", "api"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put the CUDA toolkit on PATH)")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "spmv.h")]
    return max(os.path.getmtime(p) for p in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every CUDA unit for sm_103a and link the shared library.  Returns its path."""
    if not force and not extra_flags and os.path.exists(LIB) and os.path.getmtime(LIB) >= _sources():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + list(extra_flags or [])
    procs = []
    for u in UNITS:
        obj = os.path.join(BUILD, u + ".o")
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, u + ".cu"), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = []
    for u, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(f"--- {u}.cu ---\n{out}")
        elif verbose and out.strip():
            print(out, file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [os.path.join(BUILD, u + ".o") for u in UNITS]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
