"""Build the CUDA library liblbfluct.so in-tree for sm_103a (GB300).

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked
into paper_0803_2826_gb300/liblbfluct.so.  Objects go to _build/ (ignored).
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
OUT = os.path.join(PKG, "liblbfluct.so")
BUILD = os.path.join(ROOT, "_build")
# the index-checking variant (-DLB_DEBUG_BOUNDS): every population pull and
# store and every particle spread index is tested against its array first; a
# violation sets LB_DERR_BOUNDS in the handle's error word and skips the access
OUT_BOUNDS = os.path.join(PKG, "liblbfluct_bounds.so")
BUILD_BOUNDS = os.path.join(ROOT, "_build", "bounds")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbfluct.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


# the files that define the fused stream-collide kernel
STREAM_COLLIDE_FILES = ("d3q19.cuh", "f32x2.cuh", "stream_collide.cuh", "sc_f32.cu", "sc_f16.cu", "sc_bf16.cu",
                        "step_args.h")


def source_hash(files=None) -> str:
    """SHA-1 over the library sources, or over the named files of csrc/ (to
    tie profiles to the code they measured)."""
    import hashlib
    h = hashlib.sha1()
    deps = _deps() if files is None else [os.path.join(CSRC, f) for f in files]
    for f in sorted(deps):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def up_to_date(out: str = OUT) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug_bounds: bool = False) -> str:
    """Compile and link liblbfluct.so (or, with debug_bounds, the index-checking
    liblbfluct_bounds.so) unless it is newer than every source."""
    out = OUT_BOUNDS if debug_bounds else OUT
    bdir = BUILD_BOUNDS if debug_bounds else BUILD
    flags = list(extra_flags) + (["-DLB_DEBUG_BOUNDS"] if debug_bounds else [])
    if not force and up_to_date(out):
        return out
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug_bounds="--bounds" in sys.argv))
