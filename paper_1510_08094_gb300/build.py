"""Build the CUDA library in-tree: _build/libsphere_poisson.so (sm_103a only).

Run as `python -m paper_1510_08094_gb300.build` or through __graft_entry__.build().
The library is rebuilt when any source under csrc/ or include/ is newer than it.
"""

from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB_NAME = "libsphere_poisson.so"
LIB_PATH = os.path.join(BUILD, LIB_NAME)
SOURCES = ["sphere_poisson.cu", "pipe_probe.cu", "k_f64.cu", "k_f32.cu", "k_dd.cu", "k_batched_dd.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed ({res.returncode}): {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        print(res.stderr, file=sys.stderr)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if needed and return its path.  The translation
    units compile in parallel, then link into one shared library."""
    if not force and up_to_date():
        return LIB_PATH
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    if verbose:
        flags.append("-Xptxas=-v")
    tag = f"{os.getpid()}"
    objs = [os.path.join(BUILD, os.path.splitext(s)[0] + f".{tag}.o") for s in SOURCES]
    jobs = [[nvcc] + flags + ["-c", os.path.join(CSRC, s), "-o", o] for s, o in zip(SOURCES, objs)]
    tmp = LIB_PATH + f".tmp{tag}"
    try:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for fut in [ex.submit(_run, j, verbose) for j in jobs]:
                fut.result()
        _run([nvcc, ARCH, "-shared", "-o", tmp] + objs, verbose)
        os.replace(tmp, LIB_PATH)
    finally:
        for o in objs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
