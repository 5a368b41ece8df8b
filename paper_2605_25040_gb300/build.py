"""Builds libcafs.so (the CUDA library behind the C ABI in include/cafs.h).

Every translation unit under csrc/ is compiled with nvcc for sm_103a only,
in parallel, then linked into ``paper_2605_25040_gb300/libcafs.so``.  The
object files go to ``paper_2605_25040_gb300/_build/``.  Rebuilds happen when
a source or header is newer than the library.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcafs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcafs.so")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles and links libcafs.so; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and (res.stdout or res.stderr):
            print(res.stdout, res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, len(_sources()))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))



# The translation unit of each kernel family and the headers it includes.
KERNEL_SOURCES = {
    "pipeline_kernel": ["paper_2605_25040_gb300/csrc/cafs_pipeline.cu", "paper_2605_25040_gb300/csrc/cafs_phases.cuh",
                        "paper_2605_25040_gb300/csrc/cafs_device.cuh", "paper_2605_25040_gb300/csrc/cafs_internal.h"],
    "batch_kernel": ["paper_2605_25040_gb300/csrc/cafs_batch.cu", "paper_2605_25040_gb300/csrc/cafs_batch_host.h",
                     "paper_2605_25040_gb300/csrc/cafs_phases.cuh", "paper_2605_25040_gb300/csrc/cafs_device.cuh",
                     "paper_2605_25040_gb300/csrc/cafs_internal.h"],
}


def strip_comments(src: bytes) -> bytes:
    """C/C++ source without its // and /* */ comments (string and character
    literals kept as they are), so that a comment edit does not count as a
    change of the code."""
    out = bytearray()
    i, n = 0, len(src)
    while i < n:
        c = src[i:i + 1]
        if c in (b'"', b"'"):
            j = i + 1
            while j < n and src[j:j + 1] != c:
                j += 2 if src[j:j + 1] == b"\\" else 1
            out += src[i:j + 1]
            i = j + 1
        elif src[i:i + 2] == b"//":
            j = src.find(b"\n", i)
            i = n if j < 0 else j
        elif src[i:i + 2] == b"/*":
            j = src.find(b"*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out += c
            i += 1
    return bytes(out)


def kernel_source_hash(kernel: str, read=None) -> str:
    """SHA-256 over the sources of one kernel family (KERNEL_SOURCES), their
    comments left out.  Profile summaries record it, so that a DRAM-traffic
    figure is reported only for the code it was measured on.
    ``read(relpath) -> bytes`` substitutes another tree (e.g. a git revision)."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        data = read(rel) if read else open(os.path.join(ROOT, rel), "rb").read()
        h.update(rel.encode() + b"\0" + strip_comments(data) + b"\0")
    return h.hexdigest()
