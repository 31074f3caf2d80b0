"""Builds libdartminhash.so for sm_103a, in-tree (paper_2005_11547_gb300/_build/), and beside it
libdartminhash_checked.so: the same sources compiled with -DDM_CHECKED, whose kernels also check
their shared-memory indices and report a failed check through dm_sync_status (DM_ECHECK).

Each .cu translation unit is compiled in parallel with nvcc (both variants at once), then linked
into one shared library per variant.  The CUDA runtime is linked statically, so the libraries
need only the driver (libcuda) at run time and can be loaded (not run) on a machine without a
GPU.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libdartminhash.so")
LIB_CHECKED = os.path.join(BUILD, "libdartminhash_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-Wall", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECKED):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []

    os.makedirs(os.path.join(BUILD, "checked"), exist_ok=True)

    def compile_one(job):
        src, checked = job
        obj = os.path.join(BUILD, "checked" if checked else "", os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *(["-DDM_CHECKED"] if checked else extra), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr, checked

    jobs = [(src, checked) for checked in (False, True) for src in sources()]
    with ThreadPoolExecutor(max(1, len(jobs))) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose_ptxas:
        for _, log, checked in results:
            if not checked:
                print(log)
    for lib, checked in ((LIB, False), (LIB_CHECKED, True)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for o, _, c in results if c == checked]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
