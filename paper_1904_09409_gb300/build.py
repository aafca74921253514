"""Build libfunnel.so in-tree for sm_103a with nvcc (no cmake, no torch extension).

Each .cu file under csrc/ is compiled in parallel to an object under _build/,
then everything is linked into paper_1904_09409_gb300/libfunnel.so.  The
bounds-checked debug library libfunnel_debug.so (-DFT_DEBUG: every gather /
scatter index checked on the device, failures recorded in flag words that
ft_debug_flags reads) is built the same way into _build_debug/; build() makes
both, compiling all their units at once.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfunnel.so")
LIB_DEBUG = os.path.join(PKG, "libfunnel_debug.so")
BUILD_DEBUG = os.path.join(PKG, "_build_debug")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def build(verbose: bool = False, extra_flags=(), debug: bool = True) -> str:
    """Compile every unit of the normal library (and, with debug, of the
    bounds-checked one) in parallel, then link; returns the normal library's
    path."""
    nv = nvcc()
    srcs = sources()
    variants = [(BUILD, LIB, [])]
    if debug:
        variants.append((BUILD_DEBUG, LIB_DEBUG, ["-DFT_DEBUG"]))
    procs, objs = [], {}
    for bdir, lib, defs in variants:
        os.makedirs(bdir, exist_ok=True)
        objs[lib] = []
        for src in srcs:
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            objs[lib].append(obj)
            cmd = [nv, *ARCH, *FLAGS, *defs, *extra_flags, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"{s}:\n{o}" for s, o in failed))
    for _, lib, _ in variants:
        tmp = lib + ".tmp"
        cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs[lib], "-lcudart"]
        subprocess.run(cmd, check=True, capture_output=not verbose)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
