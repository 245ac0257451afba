"""Build libmdf.so (the CUDA library behind include/mdf.h) in-tree with nvcc.

The translation units are compiled in parallel for sm_103a only and linked
into paper_2306_08216_gb300/libmdf.so.  No CMake; a build takes about a
minute on one core per unit.  build(debug=True) makes libmdf_debug.so with
-DMDF_DEBUG: the step kernels check the index of every global load and
store that does not go through TMA, skip one outside its buffer and raise
an error word (MDF_E_CUDA at the next host wait) instead of faulting.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmdf.so")
OBJ_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libmdf_debug.so")
SOURCES = ["mdf_step.cu", "mdf_step_rho0.cu", "mdf_step_tile.cu", "mdf_step_tile16.cu", "mdf_step_tile_rho0.cu", "mdf_step_fast.cu", "mdf_step_walls.cu", "mdf_step_walls16.cu", "mdf_aux.cu", "mdf_api.cu", "mdf_batch.cu", "mdf_noalloc.cu",
           "net_kernels.cu", "net_tc.cu", "net_api.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "mdf.h"))
    return files


def _up_to_date(lib):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in _deps() + [__file__])


def _compile(src, extra, obj_dir=OBJ):
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=(), debug=False):
    """Compile and link libmdf.so (libmdf_debug.so with debug=True); returns
    its path."""
    lib, obj_dir = (LIB_DEBUG, OBJ_DEBUG) if debug else (LIB, OBJ)
    extra = list(extra) + (["-DMDF_DEBUG"] if debug else [])
    if not force and extra == (["-DMDF_DEBUG"] if debug else []) and _up_to_date(lib):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra), obj_dir), SOURCES))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else ())
    print(LIB)
