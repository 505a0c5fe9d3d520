"""Builds the CUDA library ``libceleste.so`` for sm_103a (nvcc, in-tree).

Each translation unit compiles in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``; the objects link
into ``paper_1803_00113_gb300/lib/libceleste.so``.  Rebuilds unless the
library was built here from exactly the current sources, headers, flags and
compiler: a hash of all of them is written beside the library after each
build and compared before reusing it (a library copied in from elsewhere,
whatever its timestamp, has no matching hash and is rebuilt).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "lib")
OBJ_DIR = os.path.join(ROOT, "_build", "obj")
LIB = os.path.join(OUT_DIR, "libceleste.so")
SOURCES = ["setup.cu", "pixel.cu", "epilogue.cu", "newton.cu", "step.cu", "fit.cu", "field.cu",
           "firstorder.cu", "serve.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         f"-I{INCLUDE}"]
# Per-file additions: the pixel kernels flush FP32 denormals (their exp2 of
# Gaussian tails then needs no denormal fix-up; values that small are far
# below every tolerance).  Measured slower elsewhere, so not global.
FILE_FLAGS = {"pixel.cu": ["-ftz=true"]}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "celeste.h"))
    return files


STAMP = LIB + ".sha256"


def _nvcc_version(nvcc):
    try:
        return subprocess.run([nvcc, "--version"], capture_output=True, text=True).stdout
    except OSError:
        return ""


def source_hash(nvcc=None):
    """SHA-256 over every input of the build: the sources and headers (by
    name and content), the source list, the flags and the compiler version."""
    import hashlib
    import platform
    h = hashlib.sha256()
    for f in sorted(_inputs()):
        h.update(os.path.basename(f).encode() + b"\0")
        with open(f, "rb") as fh:
            h.update(fh.read())
        h.update(b"\0")
    flags = [f for f in FLAGS if not f.startswith("-I")]
    h.update(repr((SOURCES, ARCH, flags, sorted(FILE_FLAGS.items()),
                   platform.machine())).encode())
    h.update(_nvcc_version(nvcc or _nvcc()).encode())
    return h.hexdigest()


def needs_build():
    if not os.path.exists(LIB) or not os.path.exists(STAMP):
        return True
    with open(STAMP) as f:
        return f.read().strip() != source_hash()


def build(force=False, verbose=False):
    """Compiles the library if needed; returns the path of the .so."""
    if not force and not needs_build():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    digest = source_hash(nvcc)
    if os.path.exists(STAMP):
        os.unlink(STAMP)

    def compile_one(src):
        obj = os.path.join(OBJ_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), "-c", os.path.join(CSRC, src),
               "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for (obj, log), src in zip(results, SOURCES):
            sys.stderr.write(f"== {src}\n{log}")
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
