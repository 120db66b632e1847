"""Build the CUDA library libptn.so for GB300 (sm_103a) in-tree.

Each kernel translation unit (one per model and LQR precision) is compiled by its own
nvcc process, in parallel, then linked with the C-ABI unit into
``paper_2409_20027_gb300/_build/libptn.so``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libptn.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    for c in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libptn.so")


def sources() -> list[str]:
    """All translation units; PTN_MODELS (comma list, e.g. "pendulum,cartpole") limits
    which model kernel units are built."""
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    sel = os.environ.get("PTN_MODELS")
    if sel:
        keep = set(x.strip() for x in sel.split(","))
        srcs = [s for s in srcs if not os.path.basename(s).startswith("ptn_k_")
                or os.path.basename(s).split("_")[2] in keep]
    return srcs


def _stale(obj: str, src: str, headers: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src] + headers)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, extra=None,
          out: str | None = None) -> str:
    """Compile the library; returns the path of libptn.so.

    extra: .cu files with user models (ptn_user_model.cuh), compiled with the kernel
    sources on the include path and linked into a library of their own in `out` (the
    package's objects are built as usual and reused).  PTN_USER_MODELS (comma list of
    paths) adds such files to the default build."""
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "ptn.h")]
    srcs = sources()
    objs = [os.path.join(OUT, os.path.basename(s)[:-3] + ".o") for s in srcs]
    extra = list(extra or [])
    env_extra = [x for x in os.environ.get("PTN_USER_MODELS", "").split(",") if x.strip()]
    if env_extra and out is None:
        extra += env_extra
    lib = LIB if not extra or out is None else os.path.join(out, "libptn.so")
    if extra:
        edir = out or OUT
        os.makedirs(edir, exist_ok=True)
        for e in extra:
            e = os.path.abspath(e)
            srcs.append(e)
            objs.append(os.path.join(edir, "user_" + os.path.basename(e)[:-3] + ".o"))
    todo = [(s, o) for s, o in zip(srcs, objs) if force or _stale(o, s, headers)]

    def comp(so):
        s, o = so
        cmd = [nvcc, *ARCH, *FLAGS, "-I", CSRC, "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr[-4000:]}")
        os.replace(o + ".tmp", o)
        if verbose:
            print("compiled", os.path.basename(s), flush=True)

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(comp, todo))
    # relink when anything was compiled or an object is newer than the library (another
    # build, e.g. one with user models, may have refreshed the shared objects)
    if todo or not os.path.exists(lib) or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs):
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr[-4000:])
        os.replace(tmp, lib)
    return lib


PEAKS_SRC = os.path.join(HERE, "peaks", "ptn_peaks.cu")
PEAKS_LIB = os.path.join(OUT, "libptn_peaks.so")


def build_peaks(force: bool = False) -> str:
    """Compile the FMA-throughput probe (include/ptn_peaks.h) into its own library,
    _build/libptn_peaks.so: benchmark infrastructure, not linked into libptn.so."""
    os.makedirs(OUT, exist_ok=True)
    hdr = os.path.join(HERE, "..", "include", "ptn_peaks.h")
    if force or _stale(PEAKS_LIB, PEAKS_SRC, [hdr]):
        tmp = PEAKS_LIB + f".{os.getpid()}.tmp"
        r = subprocess.run([_nvcc(), *ARCH, *FLAGS, "-shared", "-o", tmp, PEAKS_SRC, "-lcudart"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for ptn_peaks.cu:\n" + r.stderr[-4000:])
        os.replace(tmp, PEAKS_LIB)
    return PEAKS_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    print(build_peaks(force="--force" in sys.argv))
