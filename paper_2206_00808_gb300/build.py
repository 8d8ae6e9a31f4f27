"""Build libbgwchi.so (CUDA, sm_103a) in-tree with nvcc.

Each translation unit compiles in parallel; the library links the CUDA
runtime statically, so it needs only the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", os.path.join(ROOT, "include")]
# variant -> (library, object directory, extra flags); "bounds" is the
# index-checking build (-DBGW_BOUNDS=1, see csrc/bgw_bounds.cuh)
VARIANTS = {
    "default": (os.path.join(HERE, "libbgwchi.so"), os.path.join(HERE, "_build"), []),
    "bounds": (os.path.join(HERE, "libbgwchi_bounds.so"), os.path.join(HERE, "_build_bounds"), ["-DBGW_BOUNDS=1"]),
}
LIB = VARIANTS["default"][0]
LIB_BOUNDS = VARIANTS["bounds"][0]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + [os.path.join(ROOT, "include", "bgw_chi.h"), __file__]


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def build_variants(variants=("default",), force: bool = False, verbose: bool = False) -> list:
    """Compile every csrc/*.cu for sm_103a once per variant (all translation
    units of all variants in one parallel pool) and link each library;
    returns their paths."""
    todo = [v for v in variants if force or _stale(VARIANTS[v][0])]
    if todo:
        nvcc = _nvcc()
        jobs = []
        for v in todo:
            _, bdir, extra = VARIANTS[v]
            os.makedirs(bdir, exist_ok=True)
            for src in _sources():
                jobs.append((v, src, os.path.join(bdir, os.path.basename(src)[:-3] + ".o"), extra))

        def compile_one(job):
            v, src, obj, extra = job
            cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)} ({v}):\n{r.stderr}")
            return v, obj, r.stderr

        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(compile_one, jobs))
        for v in todo:
            lib = VARIANTS[v][0]
            objs = [o for vv, o, _ in results if vv == v]
            tmp = lib + f".{os.getpid()}.tmp"
            r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed ({v}):\n{r.stderr}")
            os.replace(tmp, lib)
        if verbose:
            for _, _, log in results:
                print(log)
    return [VARIANTS[v][0] for v in variants]


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile and link libbgwchi.so (or, with bounds=True, the index-checking
    libbgwchi_bounds.so); returns its path."""
    return build_variants(("bounds",) if bounds else ("default",), force, verbose)[0]


if __name__ == "__main__":
    import sys
    print(build_variants(("default", "bounds") if "--bounds" in sys.argv else ("default",),
                         force="--force" in sys.argv, verbose="-v" in sys.argv))
