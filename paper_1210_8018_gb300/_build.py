"""Compile the CUDA library liblgf.so in-tree for sm_103a: nvcc compiles the translation units in
parallel (the host code and per-type FFT units), then links them."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "liblgf.so")
SOURCES = [os.path.join(HERE, "csrc", f) for f in
           ("lgf.cu", "noalloc.cu", "fft_float.cu", "fft_double.cu", "fft_df64_planes.cu", "fft_df64_columns.cu")]
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
    """Compile every translation unit in parallel (object files under _build/), then link."""
    newest = max(os.path.getmtime(p) for p in DEPS + SOURCES)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    from concurrent.futures import ThreadPoolExecutor
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    compile_flags = [f for f in NVCC_FLAGS if f != "-shared"]

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".%d.o" % os.getpid())
        cmd = [nvcc()] + compile_flags + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = SO + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC"]
                          + objs + ["-o", tmp])
    for o in objs:
        os.remove(o)
    os.replace(tmp, SO)
    return SO
