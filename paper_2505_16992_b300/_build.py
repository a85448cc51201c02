"""Build the CUDA library in-tree for sm_103a (``libpiso.so`` next to this file).

The C ABI and the statistics kernels (piso_capi.cu) and the step kernels
(piso_kernels_{fwd,adj}_{f32,f64}.cu) are separate translation units compiled
in parallel (no relocatable device code: each unit carries its own kernels)
and linked into one shared library."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libpiso.so")
SRCS = [os.path.join(HERE, "csrc", f) for f in ("piso_capi.cu", "piso_kernels_fwd_f32.cu", "piso_kernels_fwd_f64.cu",
                                                 "piso_kernels_adj_f32.cu", "piso_kernels_adj_f64.cu")]
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


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPS + [INCLUDE])


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    import tempfile
    with tempfile.TemporaryDirectory(prefix="piso_build_") as tmpdir:
        objs, procs = [], []
        for src in SRCS:
            obj = os.path.join(tmpdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            procs.append(subprocess.Popen([nvcc()] + NVCC_FLAGS + ["-c", "-o", obj, src],
                                          stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
        logs, failed = [], False
        for p in procs:
            out, err = p.communicate()
            logs.append(out + err)
            failed |= p.returncode != 0
        if failed:
            sys.stderr.write("".join(logs))
            raise RuntimeError("nvcc failed building libpiso.so")
        tmp = LIB + ".tmp"
        res = subprocess.run([nvcc()] + LINK_FLAGS + ["-o", tmp] + objs, capture_output=True, text=True)
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
