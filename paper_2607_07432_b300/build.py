"""Build liblbmib.so (the CUDA library behind include/lbmib.h) in-tree.

Each instantiation unit compiles to its own object in parallel; objects are
rebuilt only when a source or header is newer.  Target: sm_103a only.

    python -m paper_2607_07432_b300.build [-j N] [--force]
"""
import argparse
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "liblbmib.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
CCCL = "/usr/local/cuda/include/cccl"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + CCCL,
         "-I" + os.path.join(ROOT, "include")] + ARCH


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(obj, src, hdr_mtime):
    if not os.path.exists(obj):
        return True
    m = os.path.getmtime(obj)
    return os.path.getmtime(src) > m or hdr_mtime > m


def _compile(src, obj, extra):
    cmd = [NVCC] + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    out = "\n".join(l for l in (r.stdout + r.stderr).splitlines() if "Warning: The 'compute_" not in l)
    return src, r.returncode, out


def build(jobs=None, force=False, verbose=False, ptxas_verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_mtime = max(os.path.getmtime(h) for h in _headers())
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    todo = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, s, hdr_mtime):
            todo.append((s, o))
    with cf.ThreadPoolExecutor(max_workers=jobs or os.cpu_count()) as ex:
        # the FP64 instantiations (the parity form of the path) and the
        # geometry setup: no contraction into fused multiply-adds, so that
        # every product and sum is rounded as written
        def job(t):
            base = os.path.basename(t[0])
            more = ["-fmad=false"] if ("fp64" in base or base == "api.cu") else []
            return _compile(t[0], t[1], extra + more)
        for src, rc, out in ex.map(job, todo):
            if verbose or rc or ptxas_verbose:
                sys.stdout.write("== %s\n%s\n" % (os.path.basename(src), out))
            if rc:
                raise RuntimeError("nvcc failed on %s" % src)
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [NVCC] + ARCH + ["-shared", "-cudart", "static", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=None)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-v", action="store_true")
    ap.add_argument("--ptxas", action="store_true")
    a = ap.parse_args()
    print(build(a.j, a.force, a.v, a.ptxas))
