"""Build the CUDA libraries of the package in-tree, for sm_103a only.

    python -m paper_2210_04847_gb300.build

produces ``libnacc.so`` (the marching/rendering C ABI, ``include/nacc.h``) and
``libnacc_field.so`` (the procedural stand-in field, ``include/nacc_field.h``)
next to this file. Translation units compile in parallel; a unit is rebuilt
only when it or a header is newer than its object.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + [
    "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE, "-I", CSRC,
]
# Units whose float results decide integers (which samples exist) compile with
# no multiply-add contraction; the others may contract.
NO_FMAD = {"march.cu", "prune.cu", "fused.cu"}

LIBS = {
    "libnacc.so": ["march.cu", "march_static.cu", "fused.cu", "prune.cu", "render.cu", "grid.cu", "sat.cu",
                   "device.cu"],
    "libnacc_field.so": ["field.cu"],
}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers_mtime() -> float:
    paths = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))
    ]
    return max(os.path.getmtime(p) for p in paths)


def _compile(src: str, extra=()) -> str:
    obj = os.path.join(BUILD, src.replace(".cu", ".o"))
    path = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _headers_mtime()):
        return obj
    flags = list(COMMON) + (["-fmad=false"] if src in NO_FMAD else []) + list(extra)
    cmd = [nvcc(), *flags, "-c", path, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra=()) -> dict:
    """Compile and link every library; returns {name: path}."""
    os.makedirs(BUILD, exist_ok=True)
    units = sorted({u for us in LIBS.values() for u in us})
    with ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        objs = dict(zip(units, ex.map(lambda u: _compile(u, extra), units)))
    out = {}
    for lib, us in LIBS.items():
        target = os.path.join(HERE, lib)
        deps = [objs[u] for u in us]
        if not os.path.exists(target) or os.path.getmtime(target) < max(os.path.getmtime(o) for o in deps):
            cmd = [nvcc(), *ARCH, "-shared", "-o", target + ".tmp", *deps, "-lcudart"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("link failed for %s:\n%s" % (lib, r.stderr))
            os.replace(target + ".tmp", target)
        out[lib] = target
        if verbose:
            print("built", target)
    return out


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
