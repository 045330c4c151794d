"""Build the CUDA library paper_1008_0502_b300/libseg.so for sm_103a with nvcc.

Each source in csrc/ is compiled to an object under _build/ and the objects are
linked into one shared library with the C ABI of include/seg.h.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libseg.so")
# (source, object, extra flags): maxflow.cu once per min-cut tile shape
SOURCES = [("saliency.cu", "saliency.o", []), ("prior_terms.cu", "prior_terms.o", []),
           ("maxflow.cu", "maxflow_s0.o", ["-DMF_SHAPE=0"]), ("maxflow.cu", "maxflow_s1.o", ["-DMF_SHAPE=1"]),
           ("maxflow.cu", "maxflow_s2.o", ["-DMF_SHAPE=2"]), ("maxflow_shapes.cu", "maxflow_shapes.o", []),
           ("seg_api.cu", "seg_api.o", []), ("group.cu", "group.o", []), ("mincut_static.cu", "mincut_static.o", []),
           ("diff.cu", "diff.o", [])]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "seg.h"))
    return files


def build(force: bool = False, verbose: bool = False) -> str:
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    objs, procs = [], []
    for src, o, extra in SOURCES:  # (compiled in parallel)
        obj = os.path.join(BUILD, o)
        cmd = [NVCC, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(obj)
    failed = [cmd for p, cmd in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, failed[0])
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp, *objs,
                    "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
