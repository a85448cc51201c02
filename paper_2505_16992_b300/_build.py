"""Build the CUDA library in-tree for sm_103a (``libpiso.so`` next to this file).

The C ABI and the statistics kernels (piso_capi.cu) and the step kernels
(piso_kernels_{fwd,fwdno,adj,adjno}_{f32,f64}.cu) are separate translation units
compiled in parallel (no relocatable device code: each unit carries its own
kernels) and linked into one shared library.  Objects are kept in _build/ and
a unit is recompiled only when it or a file it includes changed."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libpiso.so")
SRCS = [os.path.join(HERE, "csrc", f) for f in ("piso_capi.cu", "piso_kernels_fwd_f32.cu", "piso_kernels_fwd_f64.cu",
                                                 "piso_kernels_adj_f32.cu", "piso_kernels_adj_f64.cu",
                                                 "piso_kernels_adjno_f32.cu", "piso_kernels_adjno_f64.cu",
                                                 "piso_kernels_fwdno_f32.cu", "piso_kernels_fwdno_f64.cu")]
DEPS = [os.path.join(HERE, "csrc", f) for f in sorted(os.listdir(os.path.join(HERE, "csrc")))]
INCLUDE = os.path.join(os.path.dirname(HERE), "include", "piso.h")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + [
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "-Xptxas", "-v",
]
LINK_FLAGS = ARCH + ["-shared", "-cudart", "static"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


OBJDIR = os.path.join(HERE, "_build")     # object cache (git-ignored), so an edit rebuilds only what it touches


def _deps(src: str):
    """Files a translation unit depends on: itself and every header of csrc/;
    the C ABI unit also includes include/piso.h and the host-side .inc files."""
    csrc = os.path.join(HERE, "csrc")
    deps = [src] + [os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith(".cuh")]
    if os.path.basename(src) == "piso_capi.cu":
        deps += [INCLUDE] + [os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith(".inc")]
    return deps


def _obj(src: str) -> str:
    return os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")


def _stale(src: str) -> bool:
    o = _obj(src)
    if not os.path.exists(o):
        return True
    t = os.path.getmtime(o)
    return any(os.path.getmtime(p) > t for p in _deps(src))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPS + [INCLUDE])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    todo = [src for src in SRCS if force or _stale(src)]
    procs = []
    for src in todo:
        tmp_obj = _obj(src) + ".tmp"
        procs.append((src, tmp_obj, subprocess.Popen([nvcc()] + NVCC_FLAGS + ["-c", "-o", tmp_obj, src],
                                                     stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
    logs, failed = [], False
    for src, tmp_obj, p in procs:
        out, err = p.communicate()
        logs.append(out + err)
        with open(_obj(src)[:-2] + ".log", "w") as f:   # ptxas resource usage of the unit's kernels
            f.write(out + err)
        if p.returncode != 0:
            failed = True
        else:
            os.replace(tmp_obj, _obj(src))
    if failed:
        sys.stderr.write("".join(logs))
        raise RuntimeError("nvcc failed building libpiso.so")
    tmp = LIB + ".tmp"
    res = subprocess.run([nvcc()] + LINK_FLAGS + ["-o", tmp] + [_obj(s) for s in SRCS], capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed linking libpiso.so")
    if verbose:
        sys.stderr.write("".join(logs))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
