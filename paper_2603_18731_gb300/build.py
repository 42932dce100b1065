"""Build the CUDA library ``libqsd.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` file is compiled by its own nvcc process (in parallel),
then the objects are linked with the static CUDA runtime into one shared
library next to this file.  Files listed in ``VARIANTS`` are compiled once per
value of a preprocessor macro (one object each), so that a kernel template's
instantiations for the three precision modes compile in parallel from one
source.  Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqsd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# source file -> (macro, values): one object per value
VARIANTS = {name: ("QSD_PREC", (0, 1, 2)) for name in ("apply_inst.cu", "apply_exc_inst.cu")}
for name in ("apply_fac_inst.cu", "apply_fv_inst.cu"):
    VARIANTS[name] = ("QSD_PREC", (0, 1, 2, 3))  # 3: FP32-mixed blocks on widened x
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-Xcudafe", "--diag_suppress=177"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(HERE, "..", "include", "qsd.h")]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + _headers())


def _units():
    """(source, object name, extra flags) of every compilation unit."""
    out = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.basename(src)[:-3]
        var = VARIANTS.get(os.path.basename(src))
        if var is None:
            out.append((src, base, []))
        else:
            macro, values = var
            out.extend((src, f"{base}_{v}", [f"-D{macro}={v}"]) for v in values)
    return out


def _compile(unit, verbose: bool) -> str:
    src, name, extra = unit
    obj = os.path.join(OBJ, name + ".o")
    if _stale(obj, src):
        cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every kernel source and link ``libqsd.so``; returns its path."""
    os.makedirs(OBJ, exist_ok=True)
    units = _units()
    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(lambda u: _compile(u, verbose), units))
    # objects of sources that no longer exist are not linked
    for o in glob.glob(os.path.join(OBJ, "*.o")):
        if o not in objs:
            os.remove(o)
    if (not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs)
            or _linked_set_changed(objs)):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-fPIC", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(_LINKED, "w") as f:
            f.write("\n".join(sorted(os.path.basename(o) for o in objs)))
    return LIB


_LINKED = os.path.join(OBJ, "linked.txt")


def _linked_set_changed(objs) -> bool:
    """The library was linked from another set of objects (a unit added or
    removed without any object being newer than the library)."""
    if not os.path.exists(_LINKED):
        return True
    return open(_LINKED).read().split() != sorted(os.path.basename(o) for o in objs)


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
