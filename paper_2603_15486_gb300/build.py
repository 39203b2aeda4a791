"""In-tree build of libcf.so (the CUDA kernels + C ABI) for sm_103a.

Each .cu translation unit is compiled to an object in parallel, then linked
into ``paper_2603_15486_gb300/libcf.so``.  Objects go to ``_build/`` beside
this file; both are git-ignored.  Rebuilds only what changed.

``build(debug_bounds=True)`` (``--debug-bounds``) makes the bounds-checked
variant ``libcf_debug.so`` instead (every bucket index range-checked, see
CF_DEBUG_BOUNDS in csrc/cf_device.cuh); load it with CF_LIBRARY=<path>.
"""
from __future__ import annotations

import glob
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build", platform.machine())
LIB = os.path.join(HERE, "libcf.so")
DEBUG_BUILD = BUILD + "-debug"
DEBUG_LIB = os.path.join(HERE, "libcf_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]
# Extra nvcc flags for tuning builds (e.g. "-DCF_K_MUT=4 -DCF_MINB_MUT=3").
FLAGS += os.environ.get("CF_EXTRA_NVCC", "").split()


def _elf_matches_host(path: str) -> bool:
    """True if `path` is an ELF file built for this machine's architecture
    (x86-64 objects can travel to an Arm host with the source tree)."""
    want = {"x86_64": 0x3E, "amd64": 0x3E, "aarch64": 0xB7, "arm64": 0xB7}.get(
        platform.machine().lower())
    try:
        with open(path, "rb") as fh:
            hdr = fh.read(20)
    except OSError:
        return False
    if len(hdr) < 20 or hdr[:4] != b"\x7fELF":
        return False
    return want is None or int.from_bytes(hdr[18:20], "little") == want


def nvcc() -> str:
    c = os.environ.get("NVCC")
    if c:
        return c
    p = "/usr/local/cuda/bin/nvcc"
    return p if os.path.exists(p) else "nvcc"


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _compile(src: str, extra=(), build_dir: str = BUILD):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    newest_dep = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers()])
    if (os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep
            and _elf_matches_host(obj)):
        return obj
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    bdir = DEBUG_BUILD if debug_bounds else BUILD
    lib = DEBUG_LIB if debug_bounds else LIB
    extra = ("-DCF_DEBUG_BOUNDS=1",) if debug_bounds else ()
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if force:
        for o in glob.glob(os.path.join(bdir, "*.o")):
            os.remove(o)
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda src: _compile(src, extra, bdir), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if (not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest
            and _elf_matches_host(lib)):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          debug_bounds="--debug-bounds" in sys.argv)
