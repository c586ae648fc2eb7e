"""Build the CUDA library libba_b300.so in-tree for sm_103a (B300)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libba_b300.so")
# the same library with the index checks of -DBA_DEBUG_BOUNDS (loaded when the
# environment sets BA_DEBUG_BOUNDS=1)
LIB_DEBUG = os.path.join(HERE, "libba_b300_debug.so")
SOURCES = ["kernels.cu", "pcg.cu", "schur_explicit.cu", "adjoint.cu", "dense_tc.cu", "noalloc.cu", "gp.cu", "layout.cu", "layout_dev.cu", "ba_abi.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "--expt-relaxed-constexpr",
         "-Wno-deprecated-declarations"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "ba_b300.h"))
    return files


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    lib = LIB_DEBUG if debug_bounds else LIB
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(f) for f in _deps())
        if os.path.getmtime(lib) >= newest:
            return lib
    from concurrent.futures import ThreadPoolExecutor

    suffix = ".dbg.o" if debug_bounds else ".o"
    objs = [os.path.join(CSRC, src.replace(".cu", suffix)) for src in SOURCES]
    extra = ["-DBA_DEBUG_BOUNDS"] if debug_bounds else []

    def compile_one(i):
        cmd = [NVCC, *FLAGS, *extra, "-c", os.path.join(CSRC, SOURCES[i]), "-o", objs[i]]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        list(ex.map(compile_one, range(len(SOURCES))))
    tmp = lib + ".tmp"
    subprocess.check_call([NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp,
                           *objs, "-lcudart", "-lpthread"])
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
