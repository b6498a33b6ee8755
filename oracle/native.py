"""ctypes binding of the plain-C FP64 oracle (oracle/ocd_ref.c).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the C oracle
restates Algorithm 1 and Eq. 9 as scalar loops with one subcarrier per
OpenMP iteration, so that the CPU baseline can run on every host core.  The
test-suite checks it against the NumPy oracle (oracle/ocd.py), which is the
one pinned to the paper.  It shares no code with the CUDA library.

`build()` compiles it with the host's gcc into oracle/_build/; `ocd_detect`
builds on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import ocd as _ocd

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "ocd_ref.c")
LIBRARY = os.path.join(_HERE, "_build", "libocd_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no fused multiply-adds); returns the path."""
    if (not force and os.path.exists(LIBRARY)
            and os.path.getmtime(LIBRARY) >= os.path.getmtime(SOURCE)):
        return LIBRARY
    os.makedirs(os.path.dirname(LIBRARY), exist_ok=True)
    tmp = LIBRARY + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                    "-shared", SOURCE, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, LIBRARY)
    return LIBRARY


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_ocd_detect.argtypes = [dp, dp, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                       ctypes.c_int]
        lib.orc_ocd_detect.restype = ctypes.c_int
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    """Threads the C oracle uses when none are given (OpenMP's default)."""
    return int(_load().orc_max_threads())


def ocd_detect(H, Y, N0: float, Es: float, K: int, mode: int, order: int,
               want_llr: bool = True, threads: int = 0):
    """Algorithm 1 then Eq. 9, as oracle.ocd.ocd_detect; returns (xhat, llr or None).

    threads <= 0 uses OpenMP's default (all host cores unless OMP_NUM_THREADS
    says otherwise).
    """
    lib = _load()
    H = np.ascontiguousarray(H, dtype=np.complex128)
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    Nsc, B, U = H.shape
    T = Y.shape[1]
    if Y.shape != (Nsc, T, B):
        raise ValueError(f"Y has shape {Y.shape}, expected ({Nsc}, T, {B})")
    Q = _ocd.bits_per_symbol(order)
    z = np.empty((Nsc, T, U), dtype=np.complex128)
    llr = np.empty((Nsc, T, U, Q), dtype=np.float64) if want_llr else None
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.orc_ocd_detect(H.ctypes.data_as(dp), Y.ctypes.data_as(dp), Nsc, B, U, T,
                            float(N0), float(Es), int(K), int(mode), int(order),
                            z.ctypes.data_as(dp),
                            llr.ctypes.data_as(dp) if llr is not None else None, int(threads))
    if rc != 0:
        raise ValueError("C oracle rejected its arguments")
    return z, llr
