"""Python binding of the batched form of the C ABI (argument marshalling only).

A cell is one independent detection problem with the arguments of
`ocd_detect`; `ocd_detect_batched` detects a list of cells with the library's
persistent ticket-driven kernels, `ocd_autotune_batched` times the candidate
tiles per cell shape, and `BatchedGraph` captures one batched call into a
CUDA graph held by the library.  Outputs and the ticket-counter workspace are
allocated here with PyTorch; every step of the detection runs in the library.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native
from .api import ALGOS, _mode, _stream_handle, _storage_of, bits_per_symbol


@dataclass
class Cell:
    """One detection problem: H [Nsc, B, U], Y [Nsc, T, B] on one CUDA device
    (complex64, or 16-bit pairs as for `ocd_detect`), and its parameters.
    `xhat` / `llr` are allocated by `make_cell` (either may be None)."""
    H: torch.Tensor
    Y: torch.Tensor
    N0: float
    Es: float = 1.0
    K: int = 3
    mode: str = "mmse"
    qam_order: int = 64
    algo: str = "auto"
    xhat: torch.Tensor | None = None
    llr: torch.Tensor | None = None


def make_cell(H, Y, N0, Es=1.0, K=3, mode="mmse", qam_order=64, algo="auto",
              want_xhat=True, want_llr=True) -> Cell:
    storage, hshape = _storage_of("H", H)
    _, yshape = _storage_of("Y", Y)
    if len(hshape) != 3 or len(yshape) != 3:
        raise ValueError("H must be [Nsc, B, U] and Y [Nsc, T, B] (complex)")
    Nsc, B, U = hshape
    T = yshape[1]
    Q = bits_per_symbol(qam_order)
    dev = H.device
    x = torch.empty((Nsc, T, U), dtype=torch.complex64, device=dev) if want_xhat else None
    L = torch.empty((Nsc, T, U, Q), dtype=torch.float32, device=dev) if want_llr else None
    return Cell(H, Y, float(N0), float(Es), int(K), mode, int(qam_order), algo, x, L)


def _cell_array(cells):
    if not cells:
        return None, None
    dev = cells[0].H.device
    if dev.type != "cuda":
        raise ValueError("cells must hold CUDA tensors (the detector has no CPU path)")
    arr = (_native.CellT * len(cells))()
    for i, c in enumerate(cells):
        storage, hshape = _storage_of(f"cells[{i}].H", c.H)
        ystorage, yshape = _storage_of(f"cells[{i}].Y", c.Y)
        if ystorage != storage:
            raise TypeError(f"cells[{i}]: H and Y must use the same storage type")
        for name, t in (("H", c.H), ("Y", c.Y), ("xhat", c.xhat), ("llr", c.llr)):
            if t is not None and t.device != dev:
                raise ValueError(f"cells[{i}].{name} is on {t.device}, expected {dev}")
        if len(hshape) != 3 or len(yshape) != 3:
            raise ValueError(f"cells[{i}]: H must be [Nsc, B, U] and Y [Nsc, T, B]")
        Nsc, B, U = hshape
        T = yshape[1]
        if yshape[0] != Nsc or yshape[2] != B:
            raise ValueError(f"cells[{i}]: Y shape {yshape} does not match H {hshape}")
        Q = bits_per_symbol(c.qam_order)
        if c.xhat is not None and (c.xhat.dtype != torch.complex64 or not c.xhat.is_contiguous()
                                   or tuple(c.xhat.shape) != (Nsc, T, U)):
            raise ValueError(f"cells[{i}].xhat must be contiguous complex64 [Nsc, T, U]")
        if c.llr is not None and (c.llr.dtype != torch.float32 or not c.llr.is_contiguous()
                                  or tuple(c.llr.shape) != (Nsc, T, U, Q)):
            raise ValueError(f"cells[{i}].llr must be contiguous float32 [Nsc, T, U, Q]")
        if c.algo not in ALGOS:
            raise ValueError(f"cells[{i}]: unknown algo {c.algo!r}")
        a = arr[i]
        a.H, a.Y = c.H.data_ptr(), c.Y.data_ptr()
        a.xhat = c.xhat.data_ptr() if c.xhat is not None else None
        a.llr = c.llr.data_ptr() if c.llr is not None else None
        a.storage, a.Nsc, a.B, a.U, a.T = storage, Nsc, B, U, T
        a.N0, a.Es, a.K = c.N0, c.Es, c.K
        a.mode, a.qam_order, a.algo = _mode(c.mode), c.qam_order, ALGOS[c.algo]
    return arr, dev


def make_workspace(ncells: int, device) -> torch.Tensor:
    """Device workspace (ticket counters) for batched calls over `ncells` cells."""
    n = _native.load().ocd_batched_workspace_size(int(ncells))
    return torch.empty(max(int(n), 256), dtype=torch.uint8, device=device)


class Tune:
    """Tile choices per (B, U, T, storage), as the autotuner returns them."""

    FIELDS = ("B", "U", "T", "storage", "algo", "symbols_per_item", "lanes_per_item",
              "sc_per_ticket", "time_us")

    def __init__(self, entries=()):
        self._t = _native.TuneT()
        entries = list(entries)
        if len(entries) > _native.OCD_TUNE_MAX_ENTRIES:
            raise ValueError("too many tune entries")
        self._t.n = len(entries)
        for i, e in enumerate(entries):
            for f in self.FIELDS:
                setattr(self._t.entry[i], f, e.get(f, 0))

    @property
    def entries(self):
        return [{f: getattr(self._t.entry[i], f) for f in self.FIELDS} for i in range(self._t.n)]

    def __repr__(self):
        return f"Tune({self.entries})"


def _ws(ws, ncells, dev):
    if ws is None:
        ws = make_workspace(ncells, dev)
    if ws.device != dev or not ws.is_contiguous():
        raise ValueError("workspace must be a contiguous tensor on the cells' device")
    return ws


def ocd_detect_batched(cells, tune: Tune | None = None, workspace: torch.Tensor | None = None,
                       stream: torch.cuda.Stream | None = None):
    """Detects every cell (outputs written into cell.xhat / cell.llr); enqueued
    on `stream` (default: the current stream), nothing synchronized.  The
    workspace must not be shared with another batched call in flight."""
    lib = _native.load()
    arr, dev = _cell_array(cells)
    if arr is None:
        return cells
    ws = _ws(workspace, len(cells), dev)
    with torch.cuda.device(dev):
        st = lib.ocd_detect_batched(arr, len(cells), ctypes.byref(tune._t) if tune else None,
                                    ws.data_ptr(), ws.numel(), _stream_handle(stream))
    _native.check(st)
    return cells


def ocd_detect_batched_static(cells, tune: Tune | None = None,
                              stream: torch.cuda.Stream | None = None):
    """ocd_detect_batched for callers that cannot allocate device memory
    (the host application owns the context and its memory, or cudaMalloc's
    synchronization is not acceptable): no workspace, nothing allocated here
    or in the library (outputs must already be in the cells).  At most
    OCD_STATIC_MAX_CELLS cells; the library's counters are shared by every
    call on a device, so calls that overlap on the GPU race (use one stream).
    The first call on a device looks up the counters' address: make it
    before any stream capture."""
    lib = _native.load()
    arr, dev = _cell_array(cells)
    if arr is None:
        return cells
    with torch.cuda.device(dev):
        st = lib.ocd_detect_batched_static(arr, len(cells), ctypes.byref(tune._t) if tune else None,
                                           _stream_handle(stream))
    _native.check(st)
    return cells


def ocd_autotune_batched(cells, reps: int = 3, workspace: torch.Tensor | None = None,
                         stream: torch.cuda.Stream | None = None) -> Tune:
    """Tune table for this batch, timed on the cells' own buffers (their
    outputs are overwritten): the fastest tile per cell shape on that shape's
    cells alone, then refined on the whole batch (defaults, the 32-user
    kernel choice, tickets, arrangement per shape; a change kept only when
    the batch gets faster)."""
    lib = _native.load()
    arr, dev = _cell_array(cells)
    tune = Tune()
    if arr is None:
        return tune
    ws = _ws(workspace, len(cells), dev)
    with torch.cuda.device(dev):
        st = lib.ocd_autotune_batched(arr, len(cells), ws.data_ptr(), ws.numel(), int(reps),
                                      ctypes.byref(tune._t), _stream_handle(stream))
    _native.check(st)
    return tune


class BatchedGraph:
    """One batched call captured into a CUDA graph by the library; the cells,
    the tune table and the workspace are bound at creation."""

    def __init__(self, cells, tune: Tune | None = None, workspace: torch.Tensor | None = None):
        self._lib = _native.load()
        arr, dev = _cell_array(cells)
        if arr is None:
            raise ValueError("a graph needs at least one cell")
        self.cells = cells
        self.device = dev
        self.workspace = _ws(workspace, len(cells), dev)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            st = self._lib.ocd_graph_create_batched(
                arr, len(cells), ctypes.byref(tune._t) if tune else None,
                self.workspace.data_ptr(), self.workspace.numel(), ctypes.byref(self._h))
        _native.check(st)

    def launch(self, stream: torch.cuda.Stream | None = None):
        if not self._h:
            raise RuntimeError("graph was closed")
        with torch.cuda.device(self.device):
            st = self._lib.ocd_graph_launch(self._h, _stream_handle(stream))
        _native.check(st)

    def close(self):
        if self._h:
            st = self._lib.ocd_graph_destroy(self._h)
            self._h = ctypes.c_void_p()
            _native.check(st)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
