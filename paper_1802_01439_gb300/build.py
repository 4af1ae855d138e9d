"""Builds libdgns.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel into ``_build/`` and linked into
``_build/libdgns.so``; a unit is recompiled only when its source or any
header changed.
"""
import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libdgns.so")
SOURCES = ["api.cu", "k_laplace.cu", "k_laplace_plane.cu", "k_laplace_tma.cu", "k_laplace_split.cu", "k_tensor.cu", "k_divgrad.cu", "k_convective.cu", "k_convective_vjp.cu", "k_convective_tf64.cu",
           "k_blas.cu", "k_projection.cu", "noalloc.cu", "tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-I", os.path.join(ROOT, "include")]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdgns")
    return exe


def _headers_digest():
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + [platform.machine()]).encode())
    return h.hexdigest()


def _compile(src, hdr, verbose):
    path = os.path.join(CSRC, src)
    obj = os.path.join(OUT, src + ".o")
    stamp = obj + ".sha"
    with open(path, "rb") as fh:
        digest = hashlib.sha256(fh.read() + hdr.encode()).hexdigest()
    if os.path.exists(obj) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read() == digest:
                return obj, False
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", path, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    if verbose and r.stderr:
        print(r.stderr)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return obj, True


def build(verbose=False, jobs=None):
    """Compile (if needed) and link libdgns.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    hdr = _headers_digest()
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(lambda s: _compile(s, hdr, verbose), SOURCES))
    objs = [o for o, _ in results]
    if any(changed for _, changed in results) or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv))
