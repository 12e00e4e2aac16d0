"""Build the sm_103a shared library libsdf_b300.so in-tree with nvcc.

The library exports the C ABI of include/sdf.h.  It is compiled for
``-gencode arch=compute_103a,code=sm_103a`` only (B300).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsdf_b300.so")
SOURCES = ["sdf.cu", "warm.cu", "eig.cu"]
HEADERS = ["sdf_device.cuh", "tc_device.cuh", "host_linalg.h"]

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "--extended-lambda",
    "-Xcompiler", "-fPIC", "-Xptxas", "-v",
]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(ROOT, "include", "sdf.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile each source to an object (in parallel), then link the library."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    inc = ["-I", os.path.join(ROOT, "include")]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, *inc, "-c", "-o", obj, os.path.join(CSRC, src)]
        res = subprocess.run(cmd, capture_output=True, text=True)
        return obj, res

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    log = os.path.join(OUT_DIR, "ptxas.log")
    with open(log, "w") as f:
        for _, res in results:
            f.write(res.stdout + res.stderr)
    bad = [res for _, res in results if res.returncode != 0]
    if bad:
        sys.stderr.write("".join(r.stdout + r.stderr for r in bad))
        raise RuntimeError("nvcc failed; see " + log)
    tmp = LIB + ".tmp%d" % os.getpid()
    link = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
            *[obj for obj, _ in results]]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc link failed")
    if verbose:
        sys.stdout.write("".join(r.stderr for _, r in results))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
