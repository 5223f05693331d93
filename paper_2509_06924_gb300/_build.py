"""Builds the C-ABI library ``_build/libnr.so`` in-tree for sm_103a with
nvcc (kernels) and g++ (host API), compiling the translation units in
parallel, the arithmetic-pipe probes ``_build/libnr_peak.so`` that the
benchmark measures its roofline denominators with, and on request the
NR_DEBUG variant ``_build/debug/libnr_debug.so`` (device bounds checks that
report instead of trapping; the binding loads it when NR_DEBUG=1).  No
CMake, no torch extension machinery."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libnr.so")
PEAK_LIB = os.path.join(OUT_DIR, "libnr_peak.so")
DEBUG_LIB = os.path.join(OUT_DIR, "debug", "libnr_debug.so")
PEAK_SOURCE = "nr_peak.cu"
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["nr_mixed.cu", "nr_pair.cu", "nr_fp64.cu", "nr_noalloc.cu", "nr_profile.cu", "nr_hmc.cu", "nr_vi.cu"]
CPP_SOURCES = ["nr_api.cpp", "nr_tune.cpp"]
HEADERS = ["nr_internal.h", "nr_device.cuh"]


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home:
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _nvcc() -> str:
    return os.path.join(_cuda_home(), "bin", "nvcc")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    deps += [os.path.join(INCLUDE, "nr.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r


def build(force: bool = False, verbose: bool = False, defines=None, out: str | None = None,
          csrc: str | None = None, include: str | None = None) -> str:
    """Compile (if needed) and return the path of libnr.so.  `defines`
    (e.g. {"NR_MINB_GRAD1": 3}), `out` and a source tree (`csrc`,
    `include`) build a variant library elsewhere."""
    CSRC_ = csrc or CSRC
    INCLUDE_ = include or INCLUDE
    lib_path = out or LIB
    if not force and out is None and not _stale():
        return LIB
    out_dir = os.path.dirname(lib_path)
    os.makedirs(out_dir, exist_ok=True)
    dflags = [f"-D{k}={v}" for k, v in (defines or {}).items()]
    nvcc = _nvcc()
    inc = ["-I", INCLUDE_, "-I", CSRC_]
    jobs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        objs.append(obj)
        jobs.append([nvcc, "-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", *dflags,
                     "-Xptxas", "-v" if verbose else "-O3", *inc, "-c", os.path.join(CSRC_, src), "-o", obj])
    cuda_inc = os.path.join(_cuda_home(), "include")
    for src in CPP_SOURCES:
        obj = os.path.join(out_dir, src + ".o")
        objs.append(obj)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", *dflags, *inc, "-I", cuda_inc, "-c",
                     os.path.join(CSRC_, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(_run, jobs))
    if verbose:
        for r in results:
            print(r.stdout + r.stderr)
    tmp = lib_path + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
    os.replace(tmp, lib_path)
    return lib_path


def build_debug(force: bool = False) -> str:
    """Compile (if needed) and return the path of the NR_DEBUG library."""
    if not force and not _stale(DEBUG_LIB):
        return DEBUG_LIB
    return build(defines={"NR_DEBUG": 1}, out=DEBUG_LIB)


def build_peak(force: bool = False) -> str:
    """Compile (if needed) and return the path of libnr_peak.so."""
    src = os.path.join(CSRC, PEAK_SOURCE)
    if not force and os.path.exists(PEAK_LIB) and os.path.getmtime(PEAK_LIB) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.abspath(__file__))):
        return PEAK_LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = PEAK_LIB + ".tmp"
    _run([_nvcc(), "-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", src, "-o", tmp,
          "-cudart", "static"])
    os.replace(tmp, PEAK_LIB)
    return PEAK_LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
