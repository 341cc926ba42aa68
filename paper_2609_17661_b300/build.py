"""Build the sm_103a shared library ``libpic1d.so`` in-tree with nvcc, and
its checking build ``libpic1d_check.so`` (-DPIC1D_CHECK: the kernels test
their indexes and the host guards the slack past the particle arrays; load
it with PIC1D_LIB=.../libpic1d_check.so).

    python -m paper_2609_17661_b300.build [--verbose] [--check]
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
LIB_CHECK = os.path.join(HERE, "libpic1d_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_cmd(out=LIB, extra=()):
    return (["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
             "-I" + os.path.join(ROOT, "include"), "-o", out, *SRC, *extra])


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    out = LIB_CHECK if check else LIB
    stale = force or not os.path.exists(out) or any(os.path.getmtime(d) > os.path.getmtime(out) for d in DEPS)
    if stale:
        extra = (("-Xptxas", "-v") if verbose else ()) + (("-DPIC1D_CHECK",) if check else ())
        subprocess.check_call(nvcc_cmd(out=out, extra=extra))
    return out


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv, check="--check" in sys.argv))
