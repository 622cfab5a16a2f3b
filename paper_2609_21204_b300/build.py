"""Build libsnap_b300.so (the CUDA kernels + C ABI) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIB = PKG / "libsnap_b300.so"
BUILD = ROOT / "_build"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
          "--expt-relaxed-constexpr", "-I", str(ROOT / "include")]
# the bond sweep and the integrator must not contract a*b+c into fma
PER_FILE = {"exact.cu": ["-fmad=false"], "mh.cu": ["-fmad=false"], "observe.cu": ["-fmad=false"]}
SOURCES = ["md.cu", "nlist.cu", "exact.cu", "io.cu", "api.cu", "noalloc.cu", "mlp.cu", "mlp_api.cu", "mh.cu", "observe.cu"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (Path(c).exists() or c == "nvcc"):
            return c
    return "nvcc"


def _stale(obj: Path, src: Path) -> bool:
    if not obj.exists():
        return True
    # every header of the package and of the C ABI (the kernels share device code in .cuh files)
    deps = [src, *CSRC.glob("*.cuh"), *CSRC.glob("*.h"), *(ROOT / "include").glob("*.h")]
    return obj.stat().st_mtime < max(d.stat().st_mtime for d in deps if d.exists())


def build(verbose: bool = False, force: bool = False, extra: list[str] | None = None) -> Path:
    BUILD.mkdir(exist_ok=True)
    objs = []
    for name in SOURCES:
        src = CSRC / name
        obj = BUILD / (name + ".o")
        objs.append(obj)
        if force or _stale(obj, src):
            cmd = [nvcc(), *ARCH, *COMMON, *PER_FILE.get(name, []), *(extra or []), "-c", str(src), "-o", str(obj)]
            if verbose:
                print(" ".join(cmd), flush=True)
            subprocess.check_call(cmd)
    if force or not LIB.exists() or LIB.stat().st_mtime < max(o.stat().st_mtime for o in objs):
        tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = [nvcc(), *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
