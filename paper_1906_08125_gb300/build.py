"""Build libpicfem.so in-tree with nvcc for sm_103a (GB300).

The particle and setup kernels are compiled with ``--fmad=false`` so that the
FP64 path evaluates every expression exactly as written; the PCG and the host
code use the default contraction.  Translation units compile in parallel.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpicfem.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "--expt-relaxed-constexpr"]
UNITS = {
    "setup.cu": ["--fmad=false"],
    "particles.cu": ["--fmad=false"],
    "pcg.cu": [],
    "api.cu": [],
    "noalloc.cu": [],
    "adjoint.cu": [],
    "collide.cu": ["--fmad=false"],
    "mg.cu": [],
}
# measurement probes, compiled into the same library (not part of the cycle)
PROBES = os.path.join(HERE, "probes")
PROBE_UNITS = {"fp64_rate.cu": []}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpicfem")


def _sources():
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps += [os.path.join(PROBES, f) for f in os.listdir(PROBES)]
    deps.append(os.path.join(INCLUDE, "picfem.h"))
    deps.append(os.path.abspath(__file__))
    return deps


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _sources())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    units = [(os.path.join(CSRC, u), f) for u, f in UNITS.items()]
    units += [(os.path.join(PROBES, u), f) for u, f in PROBE_UNITS.items()]
    for path, flags in units:
        unit = os.path.basename(path)
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, *(extra or []), "-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((unit, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {u}\n{o}" for u, o in failed))
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
