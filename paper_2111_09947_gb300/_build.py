"""In-tree build of the native parts of the package.

* ``libmsgemm.so``: the CUDA library behind the C ABI of ``include/msgemm.h``,
  compiled for sm_103a only (one ``-gencode``), one object per translation
  unit, compiled in parallel and linked against the shared CUDA runtime.
* ``libsynth.so``: the seeded input generators (plain C + OpenMP).

Artefacts land next to their sources and are git-ignored.  A build is skipped
when the artefact is newer than every source it depends on.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
CSRC_DIR = os.path.join(PKG_DIR, "csrc")
INCLUDE_DIR = os.path.join(REPO_DIR, "include")
BUILD_DIR = os.path.join(PKG_DIR, "_build")

CUDA_LIB = os.path.join(PKG_DIR, "libmsgemm.so")
SYNTH_LIB = os.path.join(PKG_DIR, "libsynth.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.isdir(home):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    proc = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if proc.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + proc.stdout)


def build_synth(force: bool = False) -> str:
    src = os.path.join(PKG_DIR, "synth.c")
    if force or _stale(SYNTH_LIB, [src, __file__]):
        tmp = SYNTH_LIB + ".tmp"
        _run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"])
        os.replace(tmp, SYNTH_LIB)
    return SYNTH_LIB


def cuda_sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC_DIR, "*.cu")))


def cuda_headers() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC_DIR, "*.cuh")) + glob.glob(os.path.join(INCLUDE_DIR, "*.h")))


def build_cuda(force: bool = False, verbose_ptxas: bool = False) -> str:
    srcs = cuda_sources()
    deps = srcs + cuda_headers() + [__file__]
    if not force and not _stale(CUDA_LIB, deps):
        return CUDA_LIB
    home = _cuda_home()
    nvcc = os.path.join(home, "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc") or "nvcc"
    os.makedirs(BUILD_DIR, exist_ok=True)
    hdrs = cuda_headers() + [__file__]
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + hdrs):
            _run([nvcc, *ARCH_FLAGS, *NVCC_FLAGS, *extra, "-I", INCLUDE_DIR, "-I", CSRC_DIR,
                  "-c", src, "-o", obj])
        return obj

    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = CUDA_LIB + ".tmp"
    libdir = os.path.join(home, "lib64")
    _run([nvcc, *ARCH_FLAGS, "-shared", "-cudart", "shared", *objs, "-o", tmp,
          "-Xlinker", "-rpath", "-Xlinker", libdir])
    os.replace(tmp, CUDA_LIB)
    return CUDA_LIB


def build_all(force: bool = False) -> None:
    build_synth(force)
    build_cuda(force)
