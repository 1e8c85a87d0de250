"""Builds libpd.so for sm_103a from csrc/*.cu with nvcc (in-tree, parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "libpd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
# Per-file flags.  The step kernels are compiled without implicit multiply-add
# contraction: every fused multiply-add there is written out, so the same source
# line rounds the same way in every kernel that inlines it (one launch per step or
# several steps per launch give the same bits).
FILE_FLAGS = {"pd_step.cu": ["-fmad=false"]}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpd")
    return p


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, defines=(), lib_path: str = None, obj_dir: str = None) -> str:
    """Compiles csrc/*.cu into libpd.so.  defines: extra -D macros (tuning
    knobs); lib_path/obj_dir: build a variant elsewhere."""
    global OBJ, LIB
    OBJ = obj_dir or os.path.join(HERE, "_build")
    LIB = lib_path or os.path.join(LIB_DIR, "libpd.so")
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cu = sorted(glob.glob(os.path.join(SRC, "*.cu")))
    headers = glob.glob(os.path.join(SRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "pd.h")]
    nv = nvcc()
    jobs = []
    for f in cu:
        o = os.path.join(OBJ, os.path.basename(f)[:-3] + ".o")
        if force or _stale(o, [f] + headers):
            jobs.append((f, o))

    def run(fo):
        f, o = fo
        cmd = [nv, *ARCH, *CFLAGS, *FILE_FLAGS.get(os.path.basename(f), []), *[f"-D{d}" for d in defines], "-c", f,
               "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(f)}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg)
    objs = [os.path.join(OBJ, os.path.basename(f)[:-3] + ".o") for f in cu]
    if force or jobs or _stale(LIB, objs):
        cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nv)), "lib64")
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nv, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", f"-rpath,{cuda_lib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of libpd.so failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
