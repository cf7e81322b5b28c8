"""Build libqldpc.so in-tree (paper_2511_21660_gb300/_build/) with nvcc for sm_103a.

Every translation unit compiles in parallel; the fused kernel source is compiled
once per (message precision, max check degree, max fault degree) family.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libqldpc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-Xptxas", "-v",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]

FUSED_FAMILIES = [(0, 8, 4), (0, 16, 8), (0, 32, 8), (1, 8, 4), (1, 16, 8), (1, 32, 8)]


def _units():
    units = [("qldpc_api", "qldpc_api.cu", []), ("soft_api", "soft_api.cu", []),
             ("post_api", "post_api.cu", []), ("relay_baseline", "relay_baseline.cu", []),
             ("soft_dmem", "soft_dmem.cu", []), ("filtered_osd", "filtered_osd.cu", []),
             ("cluster_decode", "cluster_decode.cu", [])]
    for f16, dc, dv in FUSED_FAMILIES:
        units.append((f"relay_fused_{'f16' if f16 else 'f32'}_{dc}_{dv}", "relay_fused.cu",
                      [f"-DQL_MSG_F16={f16}", f"-DQL_DC={dc}", f"-DQL_DV={dv}"]))
    return units


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(ROOT, "include", "qldpc.h")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqldpc.so")
    return path


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(unit):
        name, src, defs = unit
        obj = os.path.join(BUILD, name + ".o")
        cmd = [cc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stdout}\n{r.stderr}")
        with open(os.path.join(BUILD, name + ".ptxas.txt"), "w") as f:
            f.write(r.stderr)
        return obj

    units = _units()
    with ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
