"""ctypes loader for libocd.so (the C ABI declared in include/ocd.h).

There is no fallback: if the library is missing or cannot be loaded, every
call raises.  Build it with `python -m paper_1611_08779_gb300.build`.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB_PATH

OCD_OK = 0
OCD_ERR_ARG = -1
OCD_ERR_UNSUPPORTED = -2
OCD_ERR_CUDA = -3
OCD_MMSE = 0
OCD_BOX = 1
OCD_STORE_C64 = 0
OCD_STORE_BF16 = 1
OCD_STORE_F16 = 2
OCD_ALGO_AUTO = 0
OCD_ALGO_RESIDUAL = 1
OCD_ALGO_PROJECTED = 2
OCD_ALGO_PROJECTED_WARP = 3
OCD_ALGO_PROJECTED_TC = 4
OCD_MAX_USERS = 32
OCD_MAX_ANTENNAS = 512
OCD_MAX_SWEEPS = 256
OCD_MAX_CELLS = 1024
OCD_STATIC_MAX_CELLS = 256
OCD_TUNE_MAX_ENTRIES = 64

_STATUS = {OCD_ERR_ARG: "OCD_ERR_ARG", OCD_ERR_UNSUPPORTED: "OCD_ERR_UNSUPPORTED",
           OCD_ERR_CUDA: "OCD_ERR_CUDA"}

_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_sz = ctypes.c_size_t


class CellT(ctypes.Structure):
    """ocd_cell_t of include/ocd.h."""
    _fields_ = [("H", _vp), ("Y", _vp), ("xhat", _vp), ("llr", _vp), ("storage", _i),
                ("Nsc", _i), ("B", _i), ("U", _i), ("T", _i), ("N0", _f), ("Es", _f),
                ("K", _i), ("mode", _i), ("qam_order", _i), ("algo", _i)]


class TuneEntryT(ctypes.Structure):
    """ocd_tune_entry_t of include/ocd.h."""
    _fields_ = [("B", _i), ("U", _i), ("T", _i), ("storage", _i), ("algo", _i),
                ("symbols_per_item", _i), ("lanes_per_item", _i), ("sc_per_ticket", _i),
                ("time_us", _f)]


class TuneT(ctypes.Structure):
    """ocd_tune_t of include/ocd.h."""
    _fields_ = [("n", _i), ("entry", TuneEntryT * 64)]


SIGNATURES = {
    "ocd_detect": (_i, [_vp, _vp, _i, _i, _i, _i, _f, _f, _i, _i, _i, _vp, _vp, _vp]),
    "ocd_detect_ex": (_i, [_vp, _vp, _i, _i, _i, _i, _f, _f, _i, _i, _i, _vp, _vp, _i, _vp]),
    "ocd_detect_typed": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _f, _f, _i, _i, _i, _vp, _vp, _i,
                              _vp]),
    "ocd_detect_host": (_i, [_vp, _vp, _i, _i, _i, _i, _f, _f, _i, _i, _i, _vp, _vp,
                             _vp, _vp, _vp, _vp, _i, _vp]),
    "ocd_batched_workspace_size": (_sz, [_i]),
    "ocd_detect_batched": (_i, [_vp, _i, _vp, _vp, _sz, _vp]),
    "ocd_detect_batched_static": (_i, [_vp, _i, _vp, _vp]),
    "ocd_autotune_batched": (_i, [_vp, _i, _vp, _sz, _i, _vp, _vp]),
    "ocd_graph_create_batched": (_i, [_vp, _i, _vp, _vp, _sz, ctypes.POINTER(_vp)]),
    "ocd_graph_launch": (_i, [_vp, _vp]),
    "ocd_graph_destroy": (_i, [_vp]),
    "ocd_unfolded_checkpoint_size": (_sz, [_i, _i, _i, _i, _i, _i]),
    "ocd_unfolded_workspace_size": (_sz, [_i, _i, _i]),
    "ocd_unfolded_forward": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _f, _i, _i, _i, _vp, _vp, _vp,
                                  _vp, _vp, _i, _vp]),
    "ocd_unfolded_backward": (_i, [_vp, _i, _i, _i, _i, _vp, _f, _i, _i, _i, _vp, _vp, _vp, _vp,
                                   _vp, _vp, _vp, _vp, _vp, _sz, _i, _vp]),
    "ocd_unfolded_bce_forward": (_i, [_vp, _vp, _i, _i, _i, _i, _vp, _f, _i, _i, _i, _vp, _vp,
                                      _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _i, _vp]),
    "ocd_unfolded_bce_backward": (_i, [_vp, _i, _i, _i, _i, _vp, _f, _i, _i, _i, _vp, _vp, _vp,
                                       _vp, _vp, _vp, _vp, _vp, _vp, _sz, _i, _vp]),
    "ocd_fault_status": (_i, [_i]),
    "ocd_wait_selftest": (_i, [_i, _vp]),
    "ocd_last_error": (ctypes.c_char_p, []),
    "ocd_version": (_i, []),
}


class OcdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libocd.so once and declare its prototypes."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{os.path.basename(path)} is not built; run "
                    "`python -m paper_1611_08779_gb300.build` (the detector has no CPU path)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int) -> None:
    if status != OCD_OK:
        msg = load().ocd_last_error()
        raise OcdError(status, msg.decode() if msg else "")
