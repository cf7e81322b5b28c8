"""Compile the C oracle into shared libraries under oracle/_build/.

Builds of the same source: the FP64 oracle, its single-precision mirror and the
mirror whose fault->check messages are stored in binary16 (-O2, used by the tests),
plus the FP64 oracle at -O3 (f64_O3), the build the benchmark times as its CPU
baseline.  Plain gcc, OpenMP over shots, no contraction of multiply-add
(-ffp-contract=off) and no fast-math, so the -O3 build computes the same values as
the -O2 one.  No -march=native: the same host code runs on x86 and Arm hosts.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")

VARIANTS = {
    "f64": [],
    "f32": ["-DREAL=float"],
    "f16s": ["-DREAL=float", "-DMSG_FP16"],
    "f64_O3": ["-O3"],   # the last -O flag wins
}
SOURCES = {"relay": "relay_oracle.c", "soft": "soft_dmem_oracle.c"}


def lib_path(kind: str, variant: str) -> str:
    return os.path.join(BUILD, f"liboracle_{kind}_{variant}.so")


def build(force: bool = False, quiet: bool = True) -> None:
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for kind, src in SOURCES.items():
        src_path = os.path.join(HERE, src)
        if not os.path.exists(src_path):
            continue
        variants = VARIANTS if kind == "relay" else {"f64": []}
        for var, flags in variants.items():
            out = lib_path(kind, var)
            if (not force and os.path.exists(out)
                    and os.path.getmtime(out) >= os.path.getmtime(src_path)):
                continue
            cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
                   "-ffp-contract=off", "-fno-fast-math", *flags, src_path, "-o", out + ".tmp",
                   "-lm"]
            jobs.append((cmd, out))
    procs = [(subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), o)
             for c, o in jobs]
    for p, out in procs:
        log = p.communicate()[0].decode()
        if p.returncode != 0:
            raise RuntimeError(f"oracle build failed for {out}:\n{log}")
        os.replace(out + ".tmp", out)
        if not quiet:
            print("built", out)


if __name__ == "__main__":
    build(force="--force" in sys.argv, quiet=False)
