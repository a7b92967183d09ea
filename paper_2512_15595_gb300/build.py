"""Builds libbloomgb.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units: the host API (bf_api.cu), the random-access
microbenchmark (gups.cu) and one kernel unit per (block bits, word bits)
geometry (sbf_geom.cu compiled with -DSBF_B/-DSBF_S).  They compile in
parallel; objects are reused while they are newer than every source and
header.  Output: paper_2512_15595_gb300/_build/libbloomgb.so.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libbloomgb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
GEOMETRIES = [(64, 32), (128, 32), (256, 32), (512, 32), (64, 64), (128, 64), (256, 64), (512, 64), (1024, 64)]


def nvcc() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH") or "/usr/local/cuda"
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", CSRC, "-I", INCLUDE]


def _units():
    units = [("bf_api", os.path.join(CSRC, "bf_api.cu"), []),
             ("gups", os.path.join(CSRC, "gups.cu"), []),
             ("sbf_expand", os.path.join(CSRC, "sbf_expand.cu"), []),
             ("host_stage", os.path.join(CSRC, "host_stage.cu"), []),
             ("bf_server", os.path.join(CSRC, "bf_server.cu"), []),
             ("lbf_kernels", os.path.join(CSRC, "lbf_kernels.cu"), []),
             ("lbf_tc", os.path.join(CSRC, "lbf_tc.cu"), []),
             ("tc_cost", os.path.join(CSRC, "tc_cost.cu"), [])]
    for b, s in GEOMETRIES:
        units.append((f"sbf_B{b}_S{s}", os.path.join(CSRC, "sbf_geom.cu"), [f"-DSBF_B={b}", f"-DSBF_S={s}"]))
    return units


def _newest_dep() -> float:
    deps = glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    return max(os.path.getmtime(p) for p in deps)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile (if needed) and link the library; returns its path."""
    os.makedirs(os.path.join(BUILD, "obj"), exist_ok=True)
    newest = _newest_dep()
    cmds = []
    objs = []
    for name, src, defs in _units():
        obj = os.path.join(BUILD, "obj", name + ".o")
        objs.append(obj)
        if force or ptxas_info or not os.path.exists(obj) or os.path.getmtime(obj) < newest:
            extra = ["-Xptxas", "-v"] if ptxas_info else []
            cmds.append((name, [nvcc()] + _flags() + defs + extra + ["-c", src, "-o", obj + ".tmp"], obj))

    def run(item):
        name, cmd, obj = item
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        os.replace(obj + ".tmp", obj)
        return name, p.stderr

    logs = []
    if cmds:
        with ThreadPoolExecutor(max_workers=jobs or min(len(cmds), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(run, cmds))
    if verbose or ptxas_info:
        for name, err in logs:
            print(f"== {name}\n{err}")
    if cmds or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true")
    a = ap.parse_args()
    print(build(force=a.force, ptxas_info=a.ptxas_info, verbose=True))
