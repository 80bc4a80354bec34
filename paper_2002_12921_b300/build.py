"""Build the CUDA library libvegas_b300.so (sm_103a) in-tree.

Every translation unit under csrc/ is compiled by nvcc for
``-gencode arch=compute_103a,code=sm_103a`` (in parallel, one process per
unit) and linked into ``paper_2002_12921_b300/_build/libvegas_b300.so``.
Usage: ``python -m paper_2002_12921_b300.build [--force] [--verbose] [--debug]``
(``--debug``: ``_build/debug/libvegas_b300_debug.so`` with the device checks).
``build_user_integrand`` compiles a caller's integrand file the same way.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libvegas_b300.so"
LIB = os.path.join(OUT_DIR, LIB_NAME)
DEBUG_DIR = os.path.join(OUT_DIR, "debug")
DEBUG_LIB = os.path.join(DEBUG_DIR, "libvegas_b300_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return (sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) +
            sorted(glob.glob(os.path.join(CSRC, "*.h"))) +
            [os.path.join(INCLUDE, "vegas.h"), os.path.join(INCLUDE, "vegas_user_integrand.cuh")])


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose, out_dir=OUT_DIR, extra=()):
    obj = os.path.join(out_dir, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + headers()):
        return obj
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + list(extra) + (["-Xptxas", "-v"] if verbose else []) + \
        ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(f"== {os.path.basename(src)}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link the library if any source is newer; return its path.
    debug=True builds libvegas_b300_debug.so, the same sources with the device
    checks of VEGAS_DEBUG_CHECKS (include/vegas.h, "debug build")."""
    out_dir, lib = (DEBUG_DIR, DEBUG_LIB) if debug else (OUT_DIR, LIB)
    extra = ("-DVEGAS_DEBUG_CHECKS",) if debug else ()
    os.makedirs(out_dir, exist_ok=True)
    srcs = sources()
    # a library newer than every source and header is current, whether or not
    # its object files are at hand (a copy of the tree may carry only the .so)
    if not force and not _stale(lib, srcs + headers()):
        return lib
    if force:
        for o in glob.glob(os.path.join(out_dir, "*.o")):
            os.remove(o)
    workers = max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, out_dir, extra), srcs))
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


def build_module(src: str, out: str, force: bool = False, verbose: bool = False) -> str:
    """Compile one CUDA source file into the shared library `out` with the
    library's architecture and flags (include/ on the include path), if it is
    missing or older than its source or the library's headers.  Returns `out`."""
    if force or _stale(out, [src] + headers()):
        os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + \
            ["-I", INCLUDE, "-shared", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(f"== {os.path.basename(src)}\n{r.stderr}")
        os.replace(tmp, out)
    return out


def build_user_integrand(src: str, out: str, force: bool = False, verbose: bool = False) -> str:
    """Compile a caller's integrand file (one that uses VEGAS_USER_INTEGRAND of
    include/vegas_user_integrand.cuh) into the shared library `out`."""
    return build_module(src, out, force, verbose)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                debug="--debug" in sys.argv))
