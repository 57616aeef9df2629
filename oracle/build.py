"""Compile the plain C oracle into ``oracle/liboracle.so`` (test infrastructure only).

Strict IEEE double arithmetic (no fast-math, no FMA contraction) so the oracle gives the same
numbers on x86_64 and aarch64 hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))


def build(verbose=False):
    src = os.path.join(_HERE, "fdtd_oracle.c")
    out = os.path.join(_HERE, "liboracle.so")
    if os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "fdtd_oracle.h"))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, src, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
