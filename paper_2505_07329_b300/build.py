"""Build the C-ABI libraries in-tree with nvcc for sm_103a.

    python -m paper_2505_07329_b300.build [--force] [--verbose]

  libphe.so       the production library: every source but phe_client.cu; it
                  exports no call that takes a secret key
  libphe_test.so  the same objects plus phe_client.cu compiled with
                  -DPHE_TESTING: the client-side key generation and
                  encryption that tests and the benchmark use to make inputs

Objects go to paper_2505_07329_b300/_build/.  Rebuilds only what a newer
source or header makes stale.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libphe.so")
TEST_LIB = os.path.join(PKG, "libphe_test.so")
TEST_ONLY = ("phe_client.cu",)   # compiled with -DPHE_TESTING, linked into TEST_LIB only
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--cudart", "shared",
                "-I", os.path.join(ROOT, "include")]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.hpp")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds both libraries; returns the production library's path."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs, test_objs = [], []
    todo = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        (test_objs if os.path.basename(s) in TEST_ONLY else objs).append(o)
        if force or _stale(o, [s] + hdrs):
            todo.append((s, o))

    def compile_one(so):
        s, o = so
        extra = ["-DPHE_TESTING"] if os.path.basename(s) in TEST_ONLY else []
        cmd = [NVCC] + FLAGS + extra + (["-Xptxas", "-v"] if verbose else []) + ["-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{r.stdout}\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stdout + r.stderr

    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            for log in ex.map(compile_one, todo):
                if verbose and log:
                    print(log)
    for lib, deps in ((LIB, objs), (TEST_LIB, objs + test_objs)):
        if force or todo or _stale(lib, deps):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [NVCC] + ARCH + ["-shared", "--cudart", "shared", "-o", tmp] + deps
            subprocess.run(cmd, check=True)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv))
