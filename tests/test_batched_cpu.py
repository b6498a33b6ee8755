"""Batched form, host side: the ctypes structures match include/ocd.h byte
for byte, and invalid batched arguments are rejected before any CUDA call
(no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1611_08779_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FAKE = 0x10000  # aligned, never dereferenced


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return _native.load()


LAYOUT_C = r"""
#include <stddef.h>
#include <stdio.h>
#include "ocd.h"
#define F(T, m) printf("%s.%s %zu\n", #T, #m, offsetof(T, m));
int main(void) {
  printf("ocd_cell_t %zu\n", sizeof(ocd_cell_t));
  printf("ocd_tune_entry_t %zu\n", sizeof(ocd_tune_entry_t));
  printf("ocd_tune_t %zu\n", sizeof(ocd_tune_t));
  F(ocd_cell_t, H) F(ocd_cell_t, llr) F(ocd_cell_t, storage) F(ocd_cell_t, N0)
  F(ocd_cell_t, Es) F(ocd_cell_t, K) F(ocd_cell_t, algo)
  F(ocd_tune_entry_t, sc_per_ticket) F(ocd_tune_entry_t, time_us) F(ocd_tune_t, entry)
  return 0;
}
"""


def test_structures_match_the_header(tmp_path):
    gcc = shutil.which("gcc")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build.nvcc_path())), "include")
    if gcc is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("gcc or the CUDA headers are missing")
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.check_call([gcc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc,
                           str(src), "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().split("\n") if line)
    want = {
        "ocd_cell_t": ctypes.sizeof(_native.CellT),
        "ocd_tune_entry_t": ctypes.sizeof(_native.TuneEntryT),
        "ocd_tune_t": ctypes.sizeof(_native.TuneT),
        "ocd_cell_t.H": _native.CellT.H.offset, "ocd_cell_t.llr": _native.CellT.llr.offset,
        "ocd_cell_t.storage": _native.CellT.storage.offset,
        "ocd_cell_t.N0": _native.CellT.N0.offset, "ocd_cell_t.Es": _native.CellT.Es.offset,
        "ocd_cell_t.K": _native.CellT.K.offset, "ocd_cell_t.algo": _native.CellT.algo.offset,
        "ocd_tune_entry_t.sc_per_ticket": _native.TuneEntryT.sc_per_ticket.offset,
        "ocd_tune_entry_t.time_us": _native.TuneEntryT.time_us.offset,
        "ocd_tune_t.entry": _native.TuneT.entry.offset,
    }
    assert {k: int(v) for k, v in got.items()} == want
    assert len(_native.TuneT().entry) == _native.OCD_TUNE_MAX_ENTRIES


def cell(**kw):
    c = _native.CellT()
    d = dict(H=FAKE, Y=FAKE, xhat=FAKE, llr=FAKE, storage=0, Nsc=4, B=16, U=4, T=2, N0=0.1,
             Es=1.0, K=3, mode=0, qam_order=16, algo=0)
    d.update(kw)
    for k, v in d.items():
        setattr(c, k, v)
    return c


def cells(*items):
    arr = (_native.CellT * len(items))()
    for i, c in enumerate(items):
        arr[i] = c
    return arr


def test_workspace_size(lib):
    assert lib.ocd_batched_workspace_size(0) == 0
    assert lib.ocd_batched_workspace_size(-3) == 0
    assert lib.ocd_batched_workspace_size(1) == 256
    assert lib.ocd_batched_workspace_size(64) == 256
    assert lib.ocd_batched_workspace_size(65) == 512
    assert lib.ocd_batched_workspace_size(1024) % 256 == 0


def err(lib):
    return lib.ocd_last_error().decode()


@pytest.mark.parametrize("ncells", [-1, _native.OCD_MAX_CELLS + 1])
def test_cell_count_is_checked(lib, ncells):
    arr = cells(cell())
    assert lib.ocd_detect_batched(arr, ncells, None, FAKE, 1 << 20, None) == _native.OCD_ERR_ARG
    assert "ncells" in err(lib)


def test_null_cells_and_workspace(lib):
    assert lib.ocd_detect_batched(None, 1, None, FAKE, 256, None) == _native.OCD_ERR_ARG
    arr = cells(cell())
    assert lib.ocd_detect_batched(arr, 1, None, None, 256, None) == _native.OCD_ERR_ARG
    assert lib.ocd_detect_batched(arr, 1, None, FAKE + 2, 256, None) == _native.OCD_ERR_ARG
    assert lib.ocd_detect_batched(arr, 1, None, FAKE, 64, None) == _native.OCD_ERR_ARG
    assert "smaller" in err(lib)


def test_zero_cells_is_a_no_op(lib):
    assert lib.ocd_detect_batched(None, 0, None, None, 0, None) == _native.OCD_OK


@pytest.mark.parametrize("bad,needle", [
    (dict(U=33), "U=33"), (dict(B=0), "B=0"), (dict(qam_order=8), "qam_order"),
    (dict(N0=0.0), "N0 > 0"), (dict(storage=7), "storage"), (dict(algo=9), "algo"),
    (dict(H=None), "NULL"), (dict(K=-1), "K=-1")])
def test_bad_cell_is_named(lib, bad, needle):
    arr = cells(cell(), cell(**bad), cell())
    ws = lib.ocd_batched_workspace_size(3)
    st = lib.ocd_detect_batched(arr, 3, None, FAKE, ws, None)
    assert st == _native.OCD_ERR_ARG
    assert err(lib).startswith("cell 1: ") and needle in err(lib)


def test_autotune_and_graph_arguments(lib):
    arr = cells(cell())
    tune = _native.TuneT()
    assert lib.ocd_autotune_batched(arr, 1, FAKE, 256, 3, None, None) == _native.OCD_ERR_ARG
    assert lib.ocd_autotune_batched(arr, 1, FAKE, 256, 0, ctypes.byref(tune), None) == _native.OCD_ERR_ARG
    assert lib.ocd_autotune_batched(arr, 1, FAKE, 256, 101, ctypes.byref(tune), None) == _native.OCD_ERR_ARG
    assert lib.ocd_graph_create_batched(arr, 1, None, FAKE, 256, None) == _native.OCD_ERR_ARG
    h = ctypes.c_void_p()
    bad = cells(cell(U=0))
    assert lib.ocd_graph_create_batched(bad, 1, None, FAKE, 256, ctypes.byref(h)) == _native.OCD_ERR_ARG
    assert not h
    assert lib.ocd_graph_launch(None, None) == _native.OCD_ERR_ARG
    assert lib.ocd_graph_destroy(None) == _native.OCD_OK
