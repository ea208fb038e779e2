"""Build libstokes_mg.so in-tree for sm_103a (no cmake, translation units
compiled in parallel).  Run as ``python -m paper_2407_07253_gb300.build``."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libstokes_mg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _sources():
    return {
        "fem.o": ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-c", os.path.join(CSRC, "fem.cpp")],
        "kernels.o": [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-c", os.path.join(CSRC, "kernels.cu")],
        "stokes_mg.o": [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                        "-c", os.path.join(CSRC, "stokes_mg.cu")],
        "assembly.o": [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                       "-c", os.path.join(CSRC, "assembly.cu")],
        "bkrylov.o": [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-c", os.path.join(CSRC, "bkrylov.cu")],
        "batched.o": [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-c", os.path.join(CSRC, "batched.cu")],
        "noalloc.o": [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-c", os.path.join(CSRC, "noalloc.cu")],
    }


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "stokes_mg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile the CUDA library if a source is newer than it; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    jobs = _sources()

    def run(item):
        obj, cmd = item
        full = cmd + ["-o", os.path.join(OUT, obj)]
        r = subprocess.run(full, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(full) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(run, jobs.items()))
    tmp = LIB + ".tmp"
    link = [_nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp] + [os.path.join(OUT, o) for o in objs] + \
        ["-Xlinker", "-rpath,/usr/local/cuda/lib64", "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
