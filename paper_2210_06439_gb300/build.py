"""Builds the sm_103a CUDA library liboct_hydro.so in-tree with nvcc.

The sixteen RHS kernel instances (FP64 / mixed form, four launch shapes,
conserved or primitive reconstruction) are separate translation units; they
and the host side compile in parallel to objects, which nvcc then links into
one shared library (static CUDA runtime).  Only compute_103a/sm_103a code is generated."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboct_hydro.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include", "oct_hydro.h")
UNITS = ["oct_hydro.cu", "rhs_dispatch.cu", "diag.cu"] + [f"rhs_{form}_m{mode}{rec}.cu" for rec in ("", "_prim")
                                              for form in ("fp64", "mixed") for mode in (0, 1, 2, 3)]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def _sources():
    return [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR) if f.endswith((".cu", ".cuh", ".h"))] + [INCLUDE]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles liboct_hydro.so unless it is newer than every source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in _sources()):
            return LIB
    tag = f".{os.getpid()}"
    objs, procs = [], []
    for u in UNITS:
        o = os.path.join(OUT_DIR, u.replace(".cu", "") + tag.replace(".", "_") + ".o")
        objs.append(o)
        cmd = [nvcc()] + NVCC_FLAGS + ["-c", os.path.join(SRC_DIR, u), "-o", o]
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    errors = []
    for u, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{u}:\n{out}")
        elif verbose and out:
            print(out)
    if errors:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = LIB + tag + ".so"
    r = subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
