"""Build the in-tree CUDA library ``_lib/libmfbd.so`` for sm_103a (GB300).

Compiles every translation unit under ``csrc/`` with nvcc in parallel and
links them into one shared library with the shared CUDA runtime (so the
process shares one runtime instance with PyTorch). Objects go to
``_build/`` and are rebuilt only when a source or header is newer.
"""

import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libmfbd.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = [
    "mfbd_kernels.cu", "fused_kernels.cu", "generic_kernels.cu", "generic_n48.cu", "generic_n64.cu", "generic_n96.cu",
    "generic_n128.cu", "batch_kernels.cu", "batch_kernel_v2.cu", "batch_kernel_v3.cu",
    "batch_api.cu", "frontend_kernels.cu", "ls_filter_kernels.cu", "gemm_kernels.cu", "tc_gemm.cu", "tc_grad.cu", "dict_kernels.cu",
    "mfbd_api.cu", "mfbd_noalloc.cu", "mfbd_selftest.cu", "probe_kernels.cu", "optics_host.cpp"
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def nvcc():
    env = os.environ.get("NVCC")
    if env:
        return env
    for cand in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the MOMFBD library needs the CUDA toolkit")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(src, obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + deps)


def _compile(src, ptxas_verbose):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + ["-c", src, "-o", obj]
    if ptxas_verbose and src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"] if False else []
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr))
    return obj, res.stderr


def build(force=False, verbose=False, ptxas_verbose=False):
    """Compile and link libmfbd.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    deps = _headers()
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    todo = [s for s in srcs if force or ptxas_verbose
            or _stale(s, os.path.join(BUILD, os.path.basename(s) + ".o"), deps)]
    logs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        for obj, log in ex.map(lambda s: _compile(s, ptxas_verbose), todo):
            logs.append(log)
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs]
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr))
        os.replace(tmp, LIB)
    if verbose:
        for log in logs:
            if log.strip():
                sys.stderr.write(log)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv)
    print(LIB)
