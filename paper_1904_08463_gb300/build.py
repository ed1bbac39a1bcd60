"""Build libwproj.so (the CUDA library behind the C ABI in include/wproj.h) in-tree.

Every translation unit is compiled for sm_103a only, in parallel, then linked with the
CUDA runtime (shared) and cuFFT.  Rebuilds only when a source or header is newer than
the library, and then only the objects older than their source or a header (objects built on
another kind of machine or with other flags are never reused).  build_checked() makes libwproj_checked.so, the same sources compiled with
-DWP_CHECK_BOUNDS (index checks on the kernels' main buffer accesses, read back with
wp_bounds_status); it is a test build, never the one the package loads by default.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libwproj.so")
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libwproj_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "wproj.h")]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def flags() -> list[str]:
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
                   "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def build(force: bool = False, verbose: bool = False) -> str:
    return _build(LIB, BUILD, [], force, verbose)


def build_checked(force: bool = False, verbose: bool = False) -> str:
    return _build(LIB_CHECKED, BUILD_CHECKED, ["-DWP_CHECK_BOUNDS"], force, verbose)


def _build(lib: str, build_dir: str, defines: list[str], force: bool, verbose: bool) -> str:
    if not force and not needs_build(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(nvcc))

    headers = [d for d in _deps() if not d.endswith(".cu")]
    t_headers = max(os.path.getmtime(h) for h in headers)
    # objects are reused only when they were built on this kind of machine with these flags
    stamp = os.path.join(build_dir, "stamp.txt")
    key = f"{platform.machine()} {nvcc} {' '.join(flags() + defines)}"
    if not os.path.exists(stamp) or open(stamp).read() != key:
        force = True

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, os.path.basename(src) + ".o")
        # an object newer than its source and every header is reused
        if not force and os.path.exists(obj) and os.path.getmtime(obj) > max(os.path.getmtime(src), t_headers):
            return obj
        cmd = [nvcc, *flags(), *defines, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        log = os.path.join(build_dir, os.path.basename(src) + ".ptxas.txt")
        with open(log, "w") as fh:
            fh.write(r.stderr)
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    with open(stamp, "w") as fh:
        fh.write(key)
    tmp = lib + f".{os.getpid()}.tmp"
    libdir = os.path.join(cuda_home, "lib64")
    if not os.path.isdir(libdir):
        libdir = os.path.join(cuda_home, "lib")
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lcufft",
           "-Xlinker", "-rpath", "-Xlinker", libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
