"""Builds libtrips.so (the C-ABI CUDA library) in-tree for sm_103a.

Each .cu under csrc/ is compiled by nvcc in parallel, then linked into
``paper_2401_06003_gb300/_build/libtrips.so`` with the CUDA runtime linked
statically, so loading the library needs no GPU driver.

``build(debug=True)`` makes the checking variant
``paper_2401_06003_gb300/_build_debug/libtrips_debug.so`` from the same
sources with TP_DEBUG defined: every list, pyramid, workspace and
shared-memory index the kernels compute is checked before use, and an
out-of-range one skips the access and sets TP_FLAG_BOUNDS in the status word.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libtrips.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libtrips_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtrips.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "trips.h")]


def source_hash(files=None) -> str:
    """Hash of the kernel sources' code (all of csrc/, or the named files),
    comments and whitespace removed: recorded next to measurements (ncu
    counters, accuracy reports) so that they are used only while the code they
    were taken from is unchanged."""
    import hashlib
    import re

    paths = _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) if files is None else \
        [os.path.join(CSRC, f) for f in files]
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(os.path.basename(p).encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


# the sources of the render path (projection, binning, blend, backward and their
# ABI): an accuracy report of the path is valid while these are unchanged
RENDER_PATH_FILES = ("abi.cu", "bin.cu", "blend.cu", "common.cuh")


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile and link libtrips.so (or, with debug, libtrips_debug.so) if any
    source is newer; returns its path."""
    out_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if debug:
        extra.append("-DTP_DEBUG")

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, _sources()))
    if verbose or ptxas_info:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> tuple[str, str]:
    """Both variants, compiled concurrently: (libtrips.so, libtrips_debug.so)."""
    with concurrent.futures.ThreadPoolExecutor(max_workers=2) as ex:
        rel = ex.submit(build, force)
        dbg = ex.submit(build, force, debug=True)
        return rel.result(), dbg.result()


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
