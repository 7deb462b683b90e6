"""Build the CUDA extension (sm_103a) in-tree with nvcc.

Produces ``paper_2109_06976_gb300/_build/libgrid_gb300.so``: the kernels, the
host-side model builder and the C-ABI of ``include/grid.h``. Translation units
compile in parallel; no cmake, one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgrid_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["grid_capi.cu", "grid_f32.cu", "grid_mixed.cu", "grid_f64.cu", "grid_chain.cu", "grid_lane_chain.cu", "grid_lane_chain_fdv.cu", "grid_lane_chain_id.cu", "grid_chain_part.cu", "grid_forest.cu",
           "grid_serve.cu", "grid_traj.cu", "grid_riccati.cu", "grid_peak.cu", "grid_host.cpp", "grid_nvrtc.cpp"]
# Device headers embedded for run-time compilation (name as included -> file)
EMBED = [("grid_kernel.cuh", "grid_kernel.cuh"), ("grid_phases.cuh", "grid_phases.cuh"),
         ("grid_internal.h", "grid_internal.h"), ("spatial.cuh", "spatial.cuh"),
         ("../../include/grid.h", os.path.join("..", "..", "include", "grid.h"))]
# Minimal C headers for NVRTC, which has no C library
RTC_STDDEF = """#pragma once
typedef unsigned long size_t;
typedef long ptrdiff_t;
#define offsetof(T, m) __builtin_offsetof(T, m)
"""
RTC_STDINT = """#pragma once
typedef signed char int8_t; typedef short int16_t; typedef int int32_t; typedef long long int64_t;
typedef unsigned char uint8_t; typedef unsigned short uint16_t; typedef unsigned int uint32_t;
typedef unsigned long long uint64_t; typedef unsigned long uintptr_t;
"""


def _write_embed() -> str:
    """_build/grid_embed.inc: the device headers as string literals (rewritten
    only when they change)."""
    items = [(name, open(os.path.join(CSRC, path)).read()) for name, path in EMBED]
    items += [("stddef.h", RTC_STDDEF), ("stdint.h", RTC_STDINT)]
    out = [f"static const int kEmbedCount = {len(items)};",
           "static const char* const kEmbedNames[] = {" + ", ".join(f'"{n}"' for n, _ in items) + "};",
           "static const char* const kEmbedSources[] = {"]
    for _, text in items:
        assert ")GRIDSRC\"" not in text
        out.append('R"GRIDSRC(' + text + ')GRIDSRC",')
    out.append("};")
    path = os.path.join(BUILD, "grid_embed.inc")
    new = "\n".join(out) + "\n"
    if not os.path.exists(path) or open(path).read() != new:
        with open(path, "w") as fh:
            fh.write(new)
    return path


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the extension")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "grid.h"))
    embed = _write_embed()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", *ARCH, *extra_flags]
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if _stale(obj, [path, *headers, embed]):
            cmd = [nvcc, *common, "-I", BUILD, "-c", path, "-o", obj]
            if src.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for lg in logs:
            print(lg)
    if jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc, "-shared", *ARCH, "-cudart", "static", "-o", tmp, *objs, "-ldl"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
