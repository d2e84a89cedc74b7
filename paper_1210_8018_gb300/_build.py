"""Compile the CUDA library liblgf.so in-tree for sm_103a (nvcc, one translation unit)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "liblgf.so")
SOURCES = [os.path.join(HERE, "csrc", "lgf.cu"), os.path.join(HERE, "csrc", "noalloc.cu")]
DEPS = [os.path.join(HERE, "csrc", f) for f in os.listdir(os.path.join(HERE, "csrc"))] + [
    os.path.join(os.path.dirname(HERE), "include", "lgf.h")]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force=False, verbose=False):
    newest = max(os.path.getmtime(p) for p in DEPS + SOURCES)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    tmp = SO + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + NVCC_FLAGS + SOURCES + ["-o", tmp]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO
