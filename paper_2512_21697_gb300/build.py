"""Build libdirac_gb300.so in-tree with nvcc for sm_103a (no cmake, one -gencode).

Translation units are compiled in parallel into ``_build/`` and linked into
``paper_2512_21697_gb300/libdirac_gb300.so``.  A unit is rebuilt when it or any header is newer
than its object.  ``build(debug=True)`` makes the debug variant ``libdirac_gb300_dbg.so`` (objects
in ``_build_dbg/``) with the kernels' index checks compiled in (-DDG_BOUNDS); the binding loads it
when DIRAC_BOUNDS_CHECK=1.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdirac_gb300.so")
BUILD_DBG = os.path.join(HERE, "_build_dbg")
LIB_DBG = os.path.join(HERE, "libdirac_gb300_dbg.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers():
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(ROOT, "include", "*.h")))


def _compile(src, obj, nvcc, defs=()):
    if src.endswith(".cu"):
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", *defs, "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
    else:
        cmd = [nvcc, "-O2", "-std=c++17", *defs, "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj


def build(force=False, verbose=False, debug=False):
    """Compile every CUDA/C++ unit of the library and link it; returns the .so path."""
    BUILD_, LIB_ = (BUILD_DBG, LIB_DBG) if debug else (BUILD, LIB)
    defs = ("-DDG_BOUNDS",) if debug else ()
    os.makedirs(BUILD_, exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr_time = max(os.path.getmtime(h) for h in _headers())
    jobs, objs = [], []
    for s in srcs:
        o = os.path.join(BUILD_, os.path.basename(s) + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), hdr_time):
            jobs.append((s, o))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for o in ex.map(lambda j: _compile(j[0], j[1], nvcc, defs), jobs):
                if verbose:
                    print("built", o)
    if force or jobs or not os.path.exists(LIB_) or os.path.getmtime(LIB_) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB_ + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcusolver"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB_)
    return LIB_


if __name__ == "__main__":
    print(build(verbose=True))
