"""Build libamrfd.so (CUDA, sm_103a only) in-tree next to this file.

nvcc -gencode arch=compute_103a,code=sm_103a, one object per translation unit
compiled in parallel, then linked as a shared library with the static CUDA
runtime. Outputs are git-ignored; the GPU host (aarch64) rebuilds from source.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libamrfd.so")
LIB_CHECKED = os.path.join(HERE, "libamrfd_checked.so")  # -DAMRFD_CHECKS: kernel index checks
BUILD = os.path.join(HERE, "_build")
SOURCES = ["amrfd_kernels.cu", "amrfd_adjoint.cu", "amrfd_api.cu", "amrfd_noalloc.cu", "amrfd_measure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libamrfd.so")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "amrfd.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False, extra=(), checked=False):
    """Build libamrfd.so, or with checked=True libamrfd_checked.so: the same library
    compiled with -DAMRFD_CHECKS (descriptor and index checks in the kernels that record
    AMRFD_ERR_CHECK and skip the access)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps() and not extra:
        return lib
    bdir = BUILD + ("_checked" if checked else "")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    if checked:
        extra = list(extra) + ["-DAMRFD_CHECKS"]

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + FLAGS + list(extra) + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        outs = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in outs:
            sys.stderr.write(err)
    tmp = lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in outs] + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
