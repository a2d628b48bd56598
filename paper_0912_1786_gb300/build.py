"""Compile the CUDA sources in csrc/ into the in-tree shared library libevol.so (sm_103a)."""
from __future__ import annotations

import os
import re
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libevol.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["evol_api.cu", "tree.cu", "lengths.cu", "walk.cu", "post.cu", "noalloc.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
# kernels that must compile without a local-memory stack frame (register spills): the force
# walk's single-physics variants that spilled faulted on GB300, so a spilling build of the walks
# (force walk and length-solve walk) is refused
NO_SPILL = {"walk.cu": "k_walk", "lengths.cu": "k_lengths"}


def _spilling_kernels(ptxas_log: str, prefix: str):
    """Kernels named like `prefix` with a non-zero stack frame in a `-Xptxas -v` log."""
    bad, name = [], None
    for line in ptxas_log.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            name = m.group(1)
            continue
        m = re.search(r"(\d+) bytes stack frame", line)
        if m and name and prefix in name and int(m.group(1)) > 0:
            bad.append((name, int(m.group(1))))
    return bad


def _deps():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    files.append(os.path.abspath(__file__))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Build libevol.so if any source is newer than it (or force).  Returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        check = ["-Xptxas", "-v"] if src in NO_SPILL else []
        cmd = [NVCC, *ARCH, *FLAGS, *check, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if src in NO_SPILL:
            bad = _spilling_kernels(r.stdout + r.stderr, NO_SPILL[src])
            if bad:
                raise RuntimeError(f"{src}: kernels compiled with a local-memory stack frame: {bad}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
