"""Build the GRF CUDA library (libgrf.so) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked with
the shared CUDA runtime (so the process shares one runtime with PyTorch).
A stamp file records the machine, the flags and the source hashes; an
up-to-date library is not rebuilt.
"""
from __future__ import annotations

import hashlib
import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgrf.so")
STAMP = os.path.join(BUILD, "stamp.txt")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the GRF library needs the CUDA 13 toolkit")
    return cand


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _fingerprint() -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    # the flags without the -I paths: the value must not depend on where the tree sits
    h.update(" ".join(ARCH + [f for f in NVCC_FLAGS if not f.startswith("-I")]).encode())
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode())
                    h.update(fh.read())
    return h.hexdigest()


# The sources behind each kernel kind of the 2-D Algorithm 2 step (its .cu
# files and the launch code in api.cu, with every header they include): a
# stored DRAM-traffic figure is valid while their fingerprint is unchanged.
KERNEL_SOURCES = {
    "noise_columns": ("api.cu", "fft_kernels.cu", "spec_noise.cu", "noise_fast.cu", "noise_kernels.cu"),
    "rows_c2r": ("api.cu", "fft_kernels.cu", "spec_other.cu", "c2r_tma.cu"),
}


def _include_closure(files):
    """The files and every header of this tree they include, transitively."""
    seen, todo = set(), list(files)
    while todo:
        f = todo.pop()
        if f in seen:
            continue
        path = next((os.path.join(d, f) for d in (CSRC, INCLUDE) if os.path.exists(os.path.join(d, f))), None)
        if path is None:
            continue
        seen.add(f)
        with open(path) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith("#include \""):
                    todo.append(line.split('"')[1])
    return sorted(seen)


def kernel_fingerprint(kind: str) -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(ARCH + [f for f in NVCC_FLAGS if not f.startswith("-I")]).encode())
    for f in _include_closure(KERNEL_SOURCES[kind]):
        path = next(os.path.join(d, f) for d in (CSRC, INCLUDE) if os.path.exists(os.path.join(d, f)))
        with open(path, "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(STAMP)):
        return False
    with open(STAMP) as f:
        return f.read().strip() == _fingerprint()


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link libgrf.so; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s" % (src, r.stderr[-4000:]))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr[-4000:])
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(_fingerprint())
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
