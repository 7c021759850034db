"""Builds the in-tree CUDA libraries for sm_103a with nvcc (no cmake).

  paper_2607_02236_gb300/libtacaw.so   the C-ABI library (include/tacaw.h)
  synth/libsynth.so                    the CUDA twin of the synthetic input generator

Translation units are compiled in parallel, then linked with the static CUDA runtime
so the library loads on machines without a driver (the driver is reached at run time).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    exe = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return exe


def _stale(target: str, sources) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _build_lib(srcs, headers, out, objdir, extra=(), verbose=False, force=False):
    os.makedirs(objdir, exist_ok=True)
    if not force and not _stale(out, list(srcs) + list(headers)):
        return out
    objs = []

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = out + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


def build_tacaw(verbose=False, force=False, extra=()) -> str:
    csrc = os.path.join(PKG, "csrc")
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")))
    headers = glob.glob(os.path.join(csrc, "*.cuh")) + [os.path.join(ROOT, "include", "tacaw.h")]
    return _build_lib(srcs, headers, os.path.join(PKG, "libtacaw.so"), os.path.join(PKG, "_build"),
                      extra=extra, verbose=verbose, force=force)


def build_synth(verbose=False, force=False) -> str:
    d = os.path.join(ROOT, "synth")
    srcs = [os.path.join(d, "csrc", "synth.cu")]
    return _build_lib(srcs, [], os.path.join(d, "libsynth.so"), os.path.join(d, "_build"),
                      verbose=verbose, force=force)


def build_all(verbose=False, force=False):
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        a = ex.submit(build_tacaw, verbose, force)
        b = ex.submit(build_synth, verbose, force)
        return a.result(), b.result()


if __name__ == "__main__":
    print(build_all(verbose="-v" in sys.argv, force="--force" in sys.argv))
