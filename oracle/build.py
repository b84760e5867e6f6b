"""Build the FP64 CPU oracle (test infrastructure only).

Two shared libraries are made from the same C source:
  liboracle.so      single-threaded, -O2, no FP contraction, no fast-math (the oracle proper)
  liboracle_omp.so  the same source with OpenMP over all host cores (a second CPU timing only)
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aton_oracle.c")
FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99"]


def _stale(target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t
               for f in ("aton_oracle.c", "aton_oracle.h", "build.py"))


def build(force=False, verbose=False):
    outs = []
    for name, extra in (("liboracle.so", []), ("liboracle_omp.so", ["-fopenmp"])):
        target = os.path.join(HERE, name)
        if force or _stale(target):
            cmd = ["gcc", *FLAGS, *extra, "-o", target, SRC, "-lm"]
            if verbose:
                print(" ".join(cmd))
            subprocess.run(cmd, check=True)
        outs.append(target)
    return outs


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
