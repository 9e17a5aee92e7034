"""Build the FRKC2 CUDA library in-tree: ``paper_1702_03818_gb300/_lib/libfrkc2.so``.

Every source under ``csrc/`` is compiled by nvcc for sm_103a only (one ``-gencode``), the
translation units in parallel, then linked into one shared library with the static CUDA
runtime.  Usage: ``python -m paper_1702_03818_gb300.build`` (or ``build()``).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(PKG, "_lib")
LIBNAME = "libfrkc2.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the FRKC2 library needs the CUDA 13 toolkit")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _compile(nvcc, src, obj, extra):
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "-I", INCLUDE, "-I", CSRC, *extra, "-c", src, "-o", obj]
    if src.endswith(".cpp"):
        cmd[1:1] = ["-x", "cu"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    """Compile and link the library; returns its path.  debug=True builds the bounds-checking
    library ``libfrkc2_debug.so`` (-DFRKC2_DEBUG_BOUNDS: kernel indices checked against their
    arrays), loaded by the binding when FRKC2_DEBUG_BOUNDS=1."""
    nvcc = _nvcc()
    objdir = os.path.join(OUTDIR, "obj_debug" if debug else "obj")
    os.makedirs(objdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if debug:
        extra.append("-DFRKC2_DEBUG_BOUNDS")
    srcs = sources()
    objs = [os.path.join(objdir, os.path.basename(s) + ".o") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(lambda so: _compile(nvcc, so[0], so[1], extra), zip(srcs, objs)))
    if verbose or ptxas_info:
        for s, log in zip(srcs, logs):
            if log.strip():
                print(f"--- {os.path.basename(s)}\n{log}", file=sys.stderr)
    out = os.path.join(OUTDIR, "libfrkc2_debug.so" if debug else LIBNAME)
    tmp = out + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, ptxas_info="--ptxas" in sys.argv, debug="--debug" in sys.argv))
