"""Build the CUDA library ``_build/libdigdsmc.so`` for sm_103a with nvcc.

The translation units compile in parallel; the FP64 ones use -fmad=false so
that every FP64 expression rounds as it is written (the deterministic mode is
compared element by element with an independent implementation).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdigdsmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]
UNITS = {
    "dsmc_ops_f64.cu": ["-fmad=false"],
    "dsmc_ops_f32.cu": [],
    "dsmc_fields.cu": ["-fmad=false"],
    "dsmc_capi.cu": ["-fmad=false"],
    "dsmc_noalloc.cu": ["-fmad=false"],
    "dsmc_synth2d.cu": [],
    "dsmc_mlp.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + [
        os.path.join(os.path.dirname(HERE), "include", "dig_dsmc.h")]


def is_stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile every translation unit (in parallel) and link the shared library."""
    if not force and not is_stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nv = nvcc()
    procs = []
    objs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        cmd = [nv, *ARCH, *COMMON, *flags, *extra, "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for unit, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or (verbose and out):
            sys.stdout.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            failed.append(unit)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nv, *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
