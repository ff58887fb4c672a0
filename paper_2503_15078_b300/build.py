"""Build the in-tree shared library ``libsilg.so`` (C ABI, sm_103a) with nvcc.

Usage: ``python -m paper_2503_15078_b300.build`` (or ``build()`` from Python). Sources are
compiled in one nvcc invocation per file into ``_build/`` and linked with the static CUDA
runtime, so the library needs no CUDA shared library beyond the driver at run time.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libsilg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", f"-I{INCLUDE}", f"-I{CSRC}",
          "-Xcompiler", "-fPIC,-pthread,-Wall", "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cpp", ".cu")):
            out.append(os.path.join(CSRC, f))
    return out


def _digest(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(p.encode())
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + COMMON).encode())
    return h.hexdigest()


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile every source under csrc/ for sm_103a and link libsilg.so; returns its path.
    Skips the work when the sources and flags are unchanged since the last build."""
    nvcc = _nvcc()
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".hpp", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "silg.h"))
    digest = _digest(srcs + headers)
    stamp = os.path.join(BUILD, "libsilg.sha256")
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        if open(stamp).read().strip() == digest:
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    procs = []
    for s in srcs:
        obj = os.path.join(BUILD, os.path.basename(s) + ".o")
        cmd = [nvcc] + ARCH + COMMON + ["-c", s, "-o", obj]
        if s.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = False
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed = True
            sys.stderr.write(" ".join(cmd) + "\n" + text)
        elif verbose and text.strip():
            sys.stderr.write(text)
    if failed:
        raise RuntimeError("nvcc compilation failed")
    link = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-cudart", "static", "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout.decode(errors="replace"))
        raise RuntimeError("nvcc link failed")
    with open(stamp, "w") as fh:
        fh.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
