"""Build libfftc.so (the CUDA library behind include/fftc.h) for sm_103a.

Every ``csrc/*.cu`` file is compiled to an object in parallel, then linked into
``paper_2308_00497_gb300/_build/libfftc.so`` (CUDA runtime linked statically).
Objects are rebuilt only when their source or any ``csrc`` header is newer.

    python -m paper_2308_00497_gb300.build [--force] [--jobs N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfftc.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfftc.so")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hs.append(os.path.join(ROOT, "include", "fftc.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src: str, obj: str, extra: list[str]) -> tuple[str, str]:
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return src, r.stderr


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile and link libfftc.so; returns its path."""
    os.makedirs(os.path.join(BUILD, "obj"), exist_ok=True)
    stamp = os.path.join(BUILD, "machine.txt")
    machine = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != machine:
        force = True  # objects from another host architecture are never reused
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr = _headers_mtime()
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, "obj", os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr):
            todo.append((s, o))
    jobs = jobs or max(1, min(len(todo) or 1, os.cpu_count() or 1))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = [ex.submit(_compile, s, o, extra or []) for s, o in todo]
            for f in cf.as_completed(futs):
                src, log = f.result()
                if verbose and log:
                    print(f"== {os.path.basename(src)}\n{log}", file=sys.stderr)
    relink = bool(todo) or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)
    if relink:
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libfftc.so failed:\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    with open(stamp, "w") as f:
        f.write(machine + "\n")
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--verbose", action="store_true", help="print ptxas resource usage")
    a = ap.parse_args(argv)
    extra = ["-Xptxas", "-v"] if a.verbose else []
    print(build(force=a.force, jobs=a.jobs, verbose=a.verbose, extra=extra))


if __name__ == "__main__":
    main()
