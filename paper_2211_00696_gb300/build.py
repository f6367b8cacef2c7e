"""Builds the phikron library in-tree with nvcc for sm_103a (GB300), in two variants:

  libphikron.so          the library;
  libphikron_checked.so  the same sources compiled with -DPHIKRON_CHECKED: every global
                         access of the apply-path kernels checks its range first (a stand-in
                         for a memory checker; slow, for small cases).

Each translation unit under csrc/ is compiled in parallel (both variants in one pool) to an
object file in _build/ resp. _build_checked/, then linked with the CUDA runtime linked
statically.  A stamp per variant records the machine architecture, the flags and a hash of
the sources, so a copy of the tree moved to another machine (x86 -> aarch64) rebuilds.

    python -m paper_2211_00696_gb300.build [--force] [-v]
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC]


class Variant:
    def __init__(self, name: str, lib: str, build_dir: str, defines: list):
        self.name = name
        self.lib = os.path.join(HERE, lib)
        self.build_dir = os.path.join(HERE, build_dir)
        self.stamp = os.path.join(self.build_dir, "stamp.txt")
        self.defines = defines


DEFAULT = Variant("default", "libphikron.so", "_build", [])
CHECKED = Variant("checked", "libphikron_checked.so", "_build_checked", ["-DPHIKRON_CHECKED"])
VARIANTS = (DEFAULT, CHECKED)
# the default library's path and build folder (used by the binding and the tests)
LIB = DEFAULT.lib
BUILD = DEFAULT.build_dir


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the phikron library needs the CUDA toolkit to build")


def sources():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cpp")):
            out.append(os.path.join(CSRC, f))
    return out


def _digest(v: Variant) -> str:
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(ARCH_FLAGS + COMMON + v.defines).encode())
    for f in sorted(os.listdir(CSRC)) + [os.path.join("..", "..", "include", "phikron.h")]:
        p = os.path.join(CSRC, f)
        if os.path.isfile(p):
            h.update(f.encode())
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def up_to_date(v: Variant = DEFAULT) -> bool:
    if not (os.path.exists(v.lib) and os.path.exists(v.stamp)):
        return False
    with open(v.stamp) as f:
        return f.read().strip() == _digest(v)


def _compile(v: Variant, src: str, verbose: bool) -> str:
    obj = os.path.join(v.build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc()] + ARCH_FLAGS + COMMON + v.defines + ["-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + COMMON + v.defines + ["-x", "c++", "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)} ({v.name}):\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        sys.stderr.write(r.stdout + r.stderr)
    return obj


def _link(v: Variant, objs: list) -> None:
    tmp = v.lib + ".tmp"
    cmd = [nvcc()] + ARCH_FLAGS + ["-shared", "-cudart", "static", "-o", tmp] + objs + ["-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed ({v.name}):\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, v.lib)
    with open(v.stamp, "w") as f:
        f.write(_digest(v))


def build(force: bool = False, verbose: bool = False, variants=VARIANTS) -> str:
    """Builds the variants that are out of date (all of them with force); returns the default
    library's path."""
    todo = [v for v in variants if force or not up_to_date(v)]
    if todo:
        srcs = sources()
        for v in todo:
            os.makedirs(v.build_dir, exist_ok=True)
        jobs = [(v, s) for v in todo for s in srcs]
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            objs = list(ex.map(lambda j: _compile(j[0], j[1], verbose), jobs))
        for v in todo:
            _link(v, [o for (vv, _), o in zip(jobs, objs) if vv is v])
    return DEFAULT.lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
