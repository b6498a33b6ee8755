"""Build the OCD C-ABI shared library (libocd.so) in-tree for sm_103a.

Usage:  python -m paper_1611_08779_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB_NAME = "libocd.so"
LIB_PATH = os.path.join(PKG, LIB_NAME)
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["ocd_api.cu", "ocd_batched.cu", "ocd_unfolded.cu", "ocd_residual.cu", "ocd_projected.cu", "ocd_projected_tma.cu", "ocd_projected_wide.cu", "ocd_projected_lane.cu",
           "ocd_projected_h16.cu"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the OCD library needs the CUDA toolkit to build")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "ocd.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build_library(force: bool = False, verbose: bool = False, extra=None) -> str:
    """Compile libocd.so if it is missing or older than its sources."""
    if not force and up_to_date():
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    objdir = os.path.join(PKG, "_build")
    os.makedirs(objdir, exist_ok=True)
    nvcc = nvcc_path()
    common = ["-O3", "-std=c++17", *ARCH_FLAGS, "-lineinfo", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, *(extra or [])]
    if verbose:
        common.append("-Xptxas=-v")
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", f".{os.getpid()}.o"))
        objs.append(obj)
        cmd = [nvcc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
    logs = []
    failed = None
    for cmd, pr in procs:
        out, _ = pr.communicate()
        logs.append(out)
        if pr.returncode != 0 and failed is None:
            failed = (cmd, out)
    if failed is not None:
        raise RuntimeError("nvcc failed:\n" + " ".join(failed[0]) + "\n" + failed[1])
    link = [nvcc, *ARCH_FLAGS, "-shared", "-o", tmp, *objs]
    proc = subprocess.run(link, capture_output=True, text=True)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    if proc.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + " ".join(link) + "\n" + proc.stdout + proc.stderr)
    if verbose:
        sys.stderr.write("".join(logs))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args(argv)
    print(build_library(force=a.force, verbose=a.verbose))


if __name__ == "__main__":
    main()
