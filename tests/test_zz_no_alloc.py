"""ocd_detect_batched_static, the entry point for callers that cannot
allocate device memory (their host application owns the context and its
memory, or cudaMalloc's synchronization is not acceptable): it keeps its
ticket counters in a library-owned device array.  Checked through the C ABI
against ocd_detect_batched on the same cells: two calls in a row give
bit-identical results (the counters are cleared on every call), nothing is
allocated, and oversized batches are rejected before any work.  This file is
collected last, and passes alone or after the rest of the suite."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import _native, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def make_cells(seed):
    cells = []
    for s in synth.mixed_cell_specs(12, seed=seed, nsc_lo=20, nsc_hi=60):
        d = synth.make_uplink(s["Nsc"], s["B"], s["U"], s["T"], s["order"], s["snr_db"], s["seed"])
        cells.append(ocd.make_cell(torch.from_numpy(d["H"]).cuda(), torch.from_numpy(d["Y"]).cuda(),
                                   d["N0"], 1.0, s["K"], s["mode"], s["order"]))
    return cells


def outputs(cells):
    return [(c.xhat.clone(), c.llr.clone()) for c in cells]


def clear(cells):
    for c in cells:
        c.xhat.fill_(float("nan"))
        c.llr.fill_(float("nan"))


def same(cells, ref):
    return all(torch.equal(c.xhat, x) and torch.equal(c.llr, L) for c, (x, L) in zip(cells, ref))


def test_static_scratch_matches_the_workspace_entry_point_twice_in_a_row():
    cells = make_cells(801)
    ocd.ocd_detect_batched(cells)
    torch.cuda.synchronize()
    ref = outputs(cells)
    for _ in range(2):
        clear(cells)
        ocd.ocd_detect_batched_static(cells)
        torch.cuda.synchronize()
        assert same(cells, ref)
    # two calls back to back on one stream, no synchronization between them
    clear(cells)
    ocd.ocd_detect_batched_static(cells)
    ocd.ocd_detect_batched_static(cells)
    torch.cuda.synchronize()
    assert same(cells, ref)
    assert ocd.fault_status(clear=False) == 0


def test_static_scratch_allocates_nothing():
    """Neither PyTorch's allocator nor the device's free memory moves across
    three calls.  The device-wide check assumes this process has the GPU to
    itself for the duration of the test (one job per GPU), so that no other
    process allocates or frees in between."""
    cells = make_cells(802)
    ocd.ocd_detect_batched_static(cells)  # first call on the device: address lookup
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        ocd.ocd_detect_batched_static(cells)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == torch_before
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_static_scratch_with_tuned_tiles_matches():
    cells = make_cells(803)
    tune = ocd.ocd_autotune_batched(cells, reps=1)
    ocd.ocd_detect_batched(cells, tune=tune)
    torch.cuda.synchronize()
    ref = outputs(cells)
    clear(cells)
    ocd.ocd_detect_batched_static(cells, tune=tune)
    torch.cuda.synchronize()
    assert same(cells, ref)


def test_oversized_batch_is_rejected_before_any_work():
    d = synth.make_uplink(2, 16, 2, 2, 16, 10.0, 804)
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    cells = [ocd.make_cell(H, Y, d["N0"], 1.0, 2, "box", 16) for _ in range(_native.OCD_STATIC_MAX_CELLS + 1)]
    for c in cells:
        c.xhat.zero_()
    with pytest.raises(ocd.OcdError, match="UNSUPPORTED"):
        ocd.ocd_detect_batched_static(cells)
    torch.cuda.synchronize()
    assert all(torch.count_nonzero(c.xhat) == 0 for c in cells)
    # exactly the limit is accepted
    ocd.ocd_detect_batched_static(cells[:_native.OCD_STATIC_MAX_CELLS])
    torch.cuda.synchronize()
    assert np.isfinite(cells[0].xhat.cpu().numpy()).all()
