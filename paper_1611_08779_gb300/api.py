"""Python binding of the OCD C ABI (argument marshalling only).

Every step of the detector runs in the CUDA library; these functions check
tensor dtypes, shapes and devices, allocate outputs with PyTorch when the
caller does not pass them, and hand raw pointers and the current CUDA stream
to the C entry points of the same names.
"""
from __future__ import annotations

import math

import torch

from . import _native

MODES = {"mmse": _native.OCD_MMSE, "box": _native.OCD_BOX,
         _native.OCD_MMSE: _native.OCD_MMSE, _native.OCD_BOX: _native.OCD_BOX}


ALGOS = {"auto": _native.OCD_ALGO_AUTO, "residual": _native.OCD_ALGO_RESIDUAL,
         "projected": _native.OCD_ALGO_PROJECTED,
         "projected_warp": _native.OCD_ALGO_PROJECTED_WARP,
         "projected_tc": _native.OCD_ALGO_PROJECTED_TC}


def bits_per_symbol(qam_order: int) -> int:
    if qam_order not in (2, 4, 16, 64, 256):
        raise ValueError(f"unsupported qam_order {qam_order}")
    return int(round(math.log2(qam_order)))


def _mode(mode) -> int:
    try:
        return MODES[mode.lower() if isinstance(mode, str) else mode]
    except KeyError:
        raise ValueError(f"unknown mode {mode!r}") from None


def _storage_of(name, t):
    """(storage code, logical complex shape) of a channel / received tensor:
    complex64 -> float32 pairs; complex32 or float16 [..., 2] -> float16
    pairs; bfloat16 [..., 2] -> bfloat16 pairs."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype == torch.complex64:
        return _native.OCD_STORE_C64, tuple(t.shape)
    if t.dtype == torch.complex32:
        return _native.OCD_STORE_F16, tuple(t.shape)
    if t.dtype in (torch.bfloat16, torch.float16) and t.dim() >= 1 and t.shape[-1] == 2:
        code = _native.OCD_STORE_BF16 if t.dtype == torch.bfloat16 else _native.OCD_STORE_F16
        return code, tuple(t.shape[:-1])
    raise TypeError(f"{name}: expected complex64, complex32 or a bfloat16/float16 [..., 2] "
                    f"tensor, got {t.dtype} {tuple(t.shape)}")


def _check_c64(name, t, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.complex64:
        raise TypeError(f"{name} must be complex64, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def ocd_detect(H: torch.Tensor, Y: torch.Tensor, N0: float, Es: float = 1.0, K: int = 3,
               mode="mmse", qam_order: int = 64, xhat: torch.Tensor | None = None,
               llr: torch.Tensor | None = None, want_xhat: bool = True, want_llr: bool = True,
               algo: str = "auto", stream: torch.cuda.Stream | None = None):
    """OCD equalization (Algorithm 1) and max-log LLRs (Eq. 9) on the GPU.

    H: [Nsc, B, U] and Y: [Nsc, T, B] complex on one CUDA device, both
    complex64, or both 16-bit pairs (complex32, or bfloat16 / float16 with a
    trailing dimension of 2 holding (re, im)).
    `algo` picks the arrangement ("auto", "residual", "projected",
    "projected_warp" or "projected_tc"; see
    include/ocd.h).  Returns (xhat complex64 [Nsc, T, U] or None,
    llr float32 [Nsc, T, U, Q] or None).
    The work is enqueued on `stream` (default: the current stream); nothing
    is synchronized.
    """
    lib = _native.load()
    storage, hshape = _storage_of("H", H)
    ystorage, yshape = _storage_of("Y", Y)
    dev = H.device
    if dev.type != "cuda":
        raise ValueError("H must be a CUDA tensor (the detector has no CPU path)")
    if Y.device != dev:
        raise ValueError(f"Y is on {Y.device}, expected {dev}")
    if ystorage != storage:
        raise TypeError("H and Y must use the same storage type")
    if len(hshape) != 3 or len(yshape) != 3:
        raise ValueError("H must be [Nsc, B, U] and Y [Nsc, T, B] (complex)")
    Nsc, B, U = hshape
    T = yshape[1]
    if yshape[0] != Nsc or yshape[2] != B:
        raise ValueError(f"Y shape {yshape} does not match H {hshape}")
    Q = bits_per_symbol(qam_order)
    if want_xhat and xhat is None:
        xhat = torch.empty((Nsc, T, U), dtype=torch.complex64, device=dev)
    if want_llr and llr is None:
        llr = torch.empty((Nsc, T, U, Q), dtype=torch.float32, device=dev)
    if xhat is not None:
        _check_c64("xhat", xhat, dev)
        if tuple(xhat.shape) != (Nsc, T, U):
            raise ValueError("xhat must be [Nsc, T, U]")
    if llr is not None:
        if llr.dtype != torch.float32 or not llr.is_contiguous() or llr.device != dev:
            raise ValueError("llr must be a contiguous float32 tensor on H's device")
        if tuple(llr.shape) != (Nsc, T, U, Q):
            raise ValueError("llr must be [Nsc, T, U, Q]")
    if algo not in ALGOS:
        raise ValueError(f"unknown algo {algo!r}")
    with torch.cuda.device(dev):
        st = lib.ocd_detect_typed(H.data_ptr(), Y.data_ptr(), storage, Nsc, B, U, T, float(N0),
                                  float(Es), int(K), _mode(mode), int(qam_order),
                                  xhat.data_ptr() if xhat is not None else None,
                                  llr.data_ptr() if llr is not None else None,
                                  ALGOS[algo], _stream_handle(stream))
    _native.check(st)
    return xhat, llr


def ocd_detect_host(H: torch.Tensor, Y: torch.Tensor, N0: float, Es: float = 1.0, K: int = 3,
                    mode="mmse", qam_order: int = 64, xhat: torch.Tensor | None = None,
                    llr: torch.Tensor | None = None, staging: dict | None = None,
                    pieces: int = 4, device: torch.device | int | None = None,
                    stream: torch.cuda.Stream | None = None):
    """Host-buffer form: H, Y and the outputs live in (preferably pinned) host
    memory; the library copies in, detects and copies out on the GPU.

    `staging` holds the device buffers {"H", "Y", "X", "L"}; pass the dict
    returned by `make_staging` to avoid allocating per call.  Results are
    valid after the stream is synchronized.
    """
    lib = _native.load()
    _check_c64("H", H)
    _check_c64("Y", Y)
    if H.device.type != "cpu" or Y.device.type != "cpu":
        raise ValueError("ocd_detect_host takes host tensors")
    Nsc, B, U = H.shape
    T = Y.shape[1]
    Q = bits_per_symbol(qam_order)
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                       (device if isinstance(device, int) else device.index))
    if staging is None:
        staging = make_staging(Nsc, B, U, T, qam_order, dev)
    if xhat is None:
        xhat = torch.empty((Nsc, T, U), dtype=torch.complex64, pin_memory=True)
    if llr is None:
        llr = torch.empty((Nsc, T, U, Q), dtype=torch.float32, pin_memory=True)
    with torch.cuda.device(dev):
        st = lib.ocd_detect_host(H.data_ptr(), Y.data_ptr(), Nsc, B, U, T, float(N0), float(Es),
                                 int(K), _mode(mode), int(qam_order),
                                 xhat.data_ptr(), llr.data_ptr(),
                                 staging["H"].data_ptr(), staging["Y"].data_ptr(),
                                 staging["X"].data_ptr(), staging["L"].data_ptr(),
                                 int(pieces), _stream_handle(stream))
    _native.check(st)
    return xhat, llr


def make_staging(Nsc: int, B: int, U: int, T: int, qam_order: int, device) -> dict:
    """Device buffers for ocd_detect_host, allocated once by the caller."""
    Q = bits_per_symbol(qam_order)
    return {
        "H": torch.empty((Nsc, B, U), dtype=torch.complex64, device=device),
        "Y": torch.empty((Nsc, T, B), dtype=torch.complex64, device=device),
        "X": torch.empty((Nsc, T, U), dtype=torch.complex64, device=device),
        "L": torch.empty((Nsc, T, U, Q), dtype=torch.float32, device=device),
    }


def fault_status(clear: bool = True) -> int:
    """Fault bits of the bulk-copy kernels (0 = no wait expired); synchronizes."""
    st = _native.load().ocd_fault_status(1 if clear else 0)
    if st < 0:
        _native.check(st)
    return st


def version() -> int:
    return _native.load().ocd_version()
