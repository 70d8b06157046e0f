"""Builds libgeomatch.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1512_06235_gb300.build        # or: python paper_1512_06235_gb300/build.py

Every translation unit is compiled in parallel, then linked with the static CUDA runtime.  A source, header or
flag change triggers a rebuild; otherwise the existing library is kept.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgeomatch.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "-Xptxas", "-O3", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]
SOURCES = ["gm_api.cu", "gm_serve.cu", "gm_bucket.cu", "gm_order.cu", "gm_match_simt.cu", "gm_match_mma.cu", "gm_match_tc.cu", "gm_noalloc.cu", "gm_tune.cu", "gm_pairs.cu", "gm_tracks.cu",
           "gm_triangulate.cu", "gm_coarse.cu", "gm_approx.cu", "gm_selftest.cu",
           "gm_stream.cu", "gm_compact.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgeomatch")


def _fingerprint() -> str:
    h = hashlib.sha256()
    h.update(" ".join(ARCH + NVCC_FLAGS + SOURCES).encode())
    files = sorted(os.listdir(CSRC)) + ["../../include/geomatch.h"]
    for name in files:
        p = os.path.normpath(os.path.join(CSRC, name))
        if os.path.isfile(p):
            with open(p, "rb") as fh:
                h.update(name.encode())
                h.update(fh.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links the library if needed; returns its path."""
    stamp = LIB + ".stamp"
    fp = _fingerprint()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == fp:
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(fp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
