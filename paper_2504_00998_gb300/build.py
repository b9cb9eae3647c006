"""Build libfe.so in-tree for sm_103a with nvcc (one -gencode, translation units in parallel).

Run as ``python -m paper_2504_00998_gb300.build`` or call :func:`build`.
"""
import concurrent.futures
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-diag-suppress", "177"]


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_lib():
    nv = os.path.realpath(_nvcc())
    root = os.path.dirname(os.path.dirname(nv))
    for d in ("lib64", os.path.join("targets", "sbsa-linux", "lib"),
              os.path.join("targets", "x86_64-linux", "lib"), "lib"):
        p = os.path.join(root, d)
        if os.path.exists(os.path.join(p, "libcublas.so")):
            return p
    return os.path.join(root, "lib64")


def _stale(obj, src, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src] + deps)


def build(verbose=False, jobs=None):
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))
    objs = []
    cmds = []
    for s in srcs:
        o = os.path.join(OUT, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if _stale(o, s, deps):
            cmds.append([nvcc] + ARCH + CFLAGS + ["-c", s, "-o", o])
    jobs = jobs or min(len(cmds) or 1, os.cpu_count() or 4)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return cmd[-1]

    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(run, cmds))
    if cmds or not os.path.exists(LIB):
        libdir = _cuda_lib()
        link = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs + [
            "-L" + libdir, "-lcublas", "-lcusolver", "-Xlinker", "-rpath=" + libdir]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
