"""Build the sm_103a shared library ``libpic1d.so`` in-tree with nvcc.

    python -m paper_2609_17661_b300.build [--verbose]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", f) for f in ("kernels.cu", "pic1d.cu", "push_stream.cu", "sort_static.cu", "surrogate.cu",
                                                   "tp_map.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", h) for h in ("pic1d_internal.h", "tc05.h", "push_device.h", "sur_mlp.h")] + \
    [os.path.join(ROOT, "include", "pic1d.h")]
LIB = os.path.join(HERE, "libpic1d.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_cmd(out=LIB, extra=()):
    return (["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
             "-I" + os.path.join(ROOT, "include"), "-o", out, *SRC, *extra])


def build(force: bool = False, verbose: bool = False) -> str:
    stale = force or not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in DEPS)
    if stale:
        cmd = nvcc_cmd(extra=("-Xptxas", "-v") if verbose else ())
        subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="--verbose" in sys.argv)
    print(LIB)
