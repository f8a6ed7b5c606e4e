"""Build liblbm.so (the C-ABI CUDA library) in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel into _build/, then
linked into paper_2201_11330_b300/liblbm.so with the CUDA runtime linked
statically.  ptxas resource usage (registers, spills) goes to
_build/ptxas.log.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "-Xptxas", "-v", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(CSRC, "*.h")) + [os.path.join(ROOT, "include", "lbm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, out: str = LIB, build_dir: str = BUILD,
          defines=()) -> str:
    """Compile every csrc/*.cu and link `out` (defines: extra -D flags)."""
    if not force and out == LIB and up_to_date():
        return LIB
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        log = open(obj + ".log", "w")
        cmd = [nvcc, *NVCC_FLAGS, *[f"-D{d}" for d in defines], *ARCH, "-c", src, "-o", obj]
        procs.append((src, obj, log, subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT)))
    failed = []
    for src, obj, log, p in procs:
        p.wait()
        log.close()
        if p.returncode != 0:
            failed.append(src)
    with open(os.path.join(build_dir, "ptxas.log"), "w") as fh:
        for src, obj, _, _ in procs:
            fh.write(open(obj + ".log").read())
    if failed:
        for src in failed:
            obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
            sys.stderr.write(open(obj + ".log").read()[-4000:])
        raise RuntimeError(f"nvcc failed for {failed}")
    objs = [os.path.join(build_dir, os.path.basename(s)[:-3] + ".o") for s in sources()]
    tmp = out + ".tmp"
    subprocess.check_call([nvcc, "-shared", *ARCH, "-o", tmp, *objs])
    os.replace(tmp, out)
    if verbose:
        print("built", out)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
