"""Build libnfftbl.so in-tree for sm_103a.

Each CUDA translation unit under csrc/ is compiled by its own nvcc process
(in parallel), then the objects are linked into one shared library next to
this file.  Nothing outside the package directory is written.

    python -m paper_2502_07155_gb300.build          # or build() from Python
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnfftbl.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "--expt-relaxed-constexpr", "-I" + os.path.join(HERE, "..", "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnfftbl")
    return path


FIXED_M = (2, 3, 4, 5, 6, 7, 8)   # must match NFFTBL_FIXED_M_LIST in plan_internal.h
GEN_DIR = os.path.join(OUT_DIR, "gen")


def generated_sources() -> list[str]:
    """One translation unit per (precision, dimension, tap count): the
    short-sum kernels are heavy templates, and splitting them lets the
    build use every core."""
    os.makedirs(GEN_DIR, exist_ok=True)
    out = []
    for ty in ("float", "double"):
        for d in (1, 2, 3):
            for w in [2 * m for m in FIXED_M] + [0]:
                path = os.path.join(GEN_DIR, f"taps_{ty}_d{d}_w{w}.cu")
                text = (f'#include "{os.path.join(CSRC, "taps.cuh")}"\n'
                        "namespace nfftbl {\n"
                        f"template nfftbl_status launch_tap_kernel<{ty}, {d}, {w}>("
                        f"nfftbl_plan_s*, const TapArgs<{ty}>&, int, size_t);\n"
                        "}\n")
                if not os.path.exists(path) or open(path).read() != text:
                    with open(path, "w") as fh:
                        fh.write(text)
                out.append(path)
    return out


def sources() -> list[str]:
    own = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    return own + generated_sources()


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) > _newest_dep(src):
        return obj
    cmd = [nvcc()] + ARCH + CFLAGS + extra + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
    if res.stderr.strip():
        sys.stderr.write(res.stderr)
    return obj


def _newest_dep(src: str) -> float:
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if not f.endswith(".cu")]
    deps.append(os.path.join(HERE, "..", "include", "nfftbl.h"))
    return max(os.path.getmtime(p) for p in deps)


def _stale(objs: list[str]) -> bool:
    if not os.path.exists(LIB):
        return True
    t_lib = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "nfftbl.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t_lib for p in deps)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    """Compile and link libnfftbl.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sources()
    if force:
        for f in os.listdir(OUT_DIR):
            if f.endswith(".o"):
                os.remove(os.path.join(OUT_DIR, f))
    elif not _stale(srcs):
        return LIB
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    print(build(force=force, verbose_ptxas="--ptxas-v" in sys.argv))
