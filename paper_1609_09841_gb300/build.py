"""Build libhermite.so in-tree for sm_103a (GB300) with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked as a
shared library next to this file.  Rebuilds only what changed (by mtime)."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhermite.so")
SOURCES = ["api.cu", "tables.cpp", "fused_f64.cu", "fused_f32.cu", "fused_f32s64.cu", "split.cu", "norms.cu", "receivers.cu", "batch.cu", "batch_api.cu", "split_static.cu", "hybrid.cu", "advect.cu", "symbol.cpp", "fused_tc.cu", "remainder.cu", "tma_map.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fno-gnu-unique: the function-local statics of template launchers (the per-device record that a
# kernel's shared-memory limit was raised) stay private to each library, also when a process loads
# the release and the debug build side by side (GNU-unique symbols would be shared between them).
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fno-gnu-unique", "--expt-relaxed-constexpr"] + \
    os.environ.get("HERMITE_NVCC_FLAGS", "").split()


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _deps():
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "hermite.h"))
    return max(os.path.getmtime(h) for h in headers)


def _compile(src, verbose, objdir=OBJ, extra=()):
    path = os.path.join(CSRC, src)
    obj = os.path.join(objdir, src + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(path), _deps()):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-I", os.path.join(ROOT, "include"), "-c", path, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "cu"] + cmd[1:]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(verbose=False, force=False, debug=False):
    """Compile and link; returns the path of libhermite.so, or with debug=True
    of libhermite_debug.so (the same sources with -DHERMITE_DEBUG: bounds
    checks in the fused kernels, objects in _build_debug)."""
    objdir = OBJ + "_debug" if debug else OBJ
    lib = os.path.join(HERE, "libhermite_debug.so") if debug else LIB
    extra = ("-DHERMITE_DEBUG",) if debug else ()
    os.makedirs(objdir, exist_ok=True)
    if force:
        for f in os.listdir(objdir):
            os.remove(os.path.join(objdir, f))
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, objdir, extra), SOURCES))
    if not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
                                  "-o", lib] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, debug="--debug" in sys.argv))
