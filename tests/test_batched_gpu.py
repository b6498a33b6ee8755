"""Batched form on the GPU: a mix of independent cells (different B, U, Nsc,
T, K, mode, alphabet, storage) detected by the persistent ticket-driven
kernels, checked cell by cell against the FP64 oracle, against the
single-problem entry point (same arrangement: bit-identical), through the
CUDA-graph wrapper and with autotuned tiles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

from .parity import assert_parity  # noqa: E402

pytestmark = pytest.mark.gpu

MODE = {"mmse": orc.MMSE, "box": orc.BOX}


def build_cells(specs, algo="auto"):
    data, cells = [], []
    for s in specs:
        d = synth.make_uplink(s["Nsc"], s["B"], s["U"], s["T"], s["order"], s["snr_db"], s["seed"])
        H = torch.from_numpy(d["H"]).cuda()
        Y = torch.from_numpy(d["Y"]).cuda()
        cells.append(ocd.make_cell(H, Y, d["N0"], 1.0, s["K"], s["mode"], s["order"],
                                   algo=s.get("algo", algo)))
        data.append(d)
    return data, cells


def check_cells(specs, data, cells, label=""):
    torch.cuda.synchronize()
    for s, d, c in zip(specs, data, cells):
        assert_parity(c.xhat.cpu().numpy(), c.llr.cpu().numpy(), d["H"], d["Y"], d["N0"], 1.0,
                      s["K"], MODE[s["mode"]], s["order"], f"{label} {s}")


def test_mixed_cells_match_the_oracle():
    specs = synth.mixed_cell_specs(12, seed=700, nsc_lo=3, nsc_hi=9)
    data, cells = build_cells(specs)
    ocd.ocd_detect_batched(cells)
    check_cells(specs, data, cells, "mixed")
    assert ocd.fault_status(clear=False) == 0


@pytest.mark.parametrize("algo", ["residual", "projected"])
def test_batched_is_bit_identical_to_the_single_problem_path(algo):
    """Each cell equals ocd_detect in the same arrangement (the batched form
    runs the single-problem kernels' per-subcarrier code, and the same
    tensor-memory kernel for the cells with 17-32 users and 9-16 symbols)."""
    specs = [s for s in synth.mixed_cell_specs(16, seed=701, nsc_lo=20, nsc_hi=60)
             if algo == "residual" or s["B"] % 2 == 0]
    data, cells = build_cells(specs, algo=algo)
    ocd.ocd_detect_batched(cells)
    torch.cuda.synchronize()
    for s, c in zip(specs, cells):
        # the batched default keeps 17-32-user cells with T <= 8 on the
        # warp-level kernel (the single-problem default takes tcgen05)
        single = algo
        if algo == "projected" and 16 < s["U"] <= 32 and s["T"] <= 8:
            single = "projected_warp"
        x, L = ocd.ocd_detect(c.H, c.Y, c.N0, 1.0, c.K, c.mode, c.qam_order, algo=single)
        torch.cuda.synchronize()
        assert torch.equal(x, c.xhat), s
        assert torch.equal(L, c.llr), s


def test_graph_replays_and_counters_reset():
    specs = synth.mixed_cell_specs(8, seed=702, nsc_lo=30, nsc_hi=80)
    data, cells = build_cells(specs)
    ocd.ocd_detect_batched(cells)
    torch.cuda.synchronize()
    ref = [(c.xhat.clone(), c.llr.clone()) for c in cells]
    g = ocd.BatchedGraph(cells)
    for _ in range(3):
        for c in cells:
            c.xhat.zero_()
            c.llr.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        for (x, L), c in zip(ref, cells):
            assert torch.equal(x, c.xhat) and torch.equal(L, c.llr)
    g.close()
    # the direct entry point again on the same workspace-sized call
    for _ in range(2):
        ocd.ocd_detect_batched(cells)
    torch.cuda.synchronize()
    for (x, L), c in zip(ref, cells):
        assert torch.equal(x, c.xhat) and torch.equal(L, c.llr)


def test_autotuned_tiles_keep_parity():
    specs = synth.mixed_cell_specs(12, seed=703, nsc_lo=40, nsc_hi=120)
    data, cells = build_cells(specs)
    tune = ocd.ocd_autotune_batched(cells, reps=1)
    shapes = {(s["B"], s["U"], s["T"]) for s in specs}
    got = {(e["B"], e["U"], e["T"]) for e in tune.entries}
    assert got == shapes
    for e in tune.entries:
        assert e["algo"] in (1, 2, 3, 4) and e["time_us"] > 0
        if e["algo"] in (3, 4):
            # the warp-level or the tcgen05 kernel: 17-32 users only
            assert 16 < e["U"] <= 32
        if e["algo"] in (2, 3, 4):
            # one symbol with U <= 8 runs the one-lane kernel: no ticket size;
            # 0 elsewhere is the default ticket size (kept by the whole-batch phase)
            lane = e["T"] == 1 and e["U"] <= 8
            assert e["U"] <= 32 and (e["sc_per_ticket"] == 0 if lane else e["sc_per_ticket"] >= 0)
        else:
            # 0: the default tile (kept by the whole-batch phase)
            assert e["symbols_per_item"] in (0, 1, 2) and e["lanes_per_item"] >= 0
    for c in cells:
        c.xhat.zero_()
        c.llr.zero_()
    ocd.ocd_detect_batched(cells, tune=tune)
    check_cells(specs, data, cells, "tuned")
    g = ocd.BatchedGraph(cells, tune=tune)
    g.launch()
    check_cells(specs, data, cells, "tuned graph")


@pytest.mark.parametrize("T", [14, 20])
def test_tune_entry_chooses_the_32_user_kernel(T):
    # a tune entry may name the warp-level or the tcgen05 kernel; results are
    # those of ocd_detect with the same kernel, and a cell the tcgen05 kernel
    # does not fit (T > 16) takes the default kernel instead
    specs = [{"B": 64, "U": 24, "T": T, "Nsc": 37, "K": 3, "mode": "box", "order": 16,
              "snr_db": 14.0, "seed": 4100},
             {"B": 64, "U": 24, "T": T, "Nsc": 21, "K": 3, "mode": "box", "order": 16,
              "snr_db": 14.0, "seed": 4101}]
    data, cells = build_cells(specs)
    for algo, name in ((3, "projected_warp"), (4, "projected_tc")):
        tune = ocd.Tune([{"B": 64, "U": 24, "T": T, "storage": 0, "algo": algo}])
        for c in cells:
            c.xhat.zero_()
            c.llr.zero_()
        ocd.ocd_detect_batched(cells, tune=tune)
        torch.cuda.synchronize()
        single = name if (name == "projected_warp" or T <= 16) else "projected"
        for c in cells:
            x, L = ocd.ocd_detect(c.H, c.Y, c.N0, c.Es, c.K, c.mode, c.qam_order, algo=single)
            assert torch.equal(x, c.xhat) and torch.equal(L, c.llr), (T, name)


def test_more_cells_than_one_launch_holds():
    # 40 cells of one kernel family: split over two launches (32 + 8)
    specs = [{"B": 16, "U": 2, "T": 3, "Nsc": 2 + i % 5, "K": 2 + i % 3,
              "mode": "box" if i % 2 else "mmse", "order": 16, "snr_db": 12.0, "seed": 900 + i}
             for i in range(40)]
    data, cells = build_cells(specs, algo="residual")
    ocd.ocd_detect_batched(cells)
    check_cells(specs, data, cells, "40 cells")
    specs2 = [dict(s, B=32, U=4, T=5) for s in specs]
    data2, cells2 = build_cells(specs2, algo="projected")
    ocd.ocd_detect_batched(cells2)
    check_cells(specs2, data2, cells2, "40 cells projected")


def test_edge_cells():
    specs = [
        {"B": 32, "U": 4, "T": 7, "Nsc": 0, "K": 3, "mode": "box", "order": 16, "snr_db": 10.0, "seed": 1},
        {"B": 33, "U": 5, "T": 6, "Nsc": 5, "K": 3, "mode": "mmse", "order": 16, "snr_db": 10.0, "seed": 2},
        {"B": 64, "U": 8, "T": 9, "Nsc": 4, "K": 0, "mode": "box", "order": 64, "snr_db": 10.0, "seed": 3},
        {"B": 16, "U": 3, "T": 4, "Nsc": 6, "K": 3, "mode": "box", "order": 2, "snr_db": 10.0, "seed": 4},
        {"B": 48, "U": 12, "T": 17, "Nsc": 3, "K": 4, "mode": "mmse", "order": 256, "snr_db": 25.0, "seed": 5},
        {"B": 512, "U": 32, "T": 2, "Nsc": 2, "K": 2, "mode": "box", "order": 4, "snr_db": 10.0, "seed": 6},
    ]
    data, cells = build_cells(specs)
    ocd.ocd_detect_batched(cells)
    check_cells(specs[1:], data[1:], cells[1:], "edge")
    # a batch of empty cells is a no-op
    ocd.ocd_detect_batched(cells[:1])
    ocd.ocd_detect_batched([])
    # the batched projected form needs the bulk-copy shape (odd B here)
    bad = [ocd.make_cell(cells[1].H, cells[1].Y, cells[1].N0, 1.0, 3, "mmse", 16, algo="projected")]
    with pytest.raises(ocd.OcdError, match="UNSUPPORTED"):
        ocd.ocd_detect_batched(bad)


def test_sixteen_bit_cells_in_a_batch():
    specs = synth.mixed_cell_specs(8, seed=704, nsc_lo=4, nsc_hi=10)
    cells, refs = [], []
    for i, s in enumerate(specs):
        d = synth.make_uplink(s["Nsc"], s["B"], s["U"], s["T"], s["order"], s["snr_db"], s["seed"])
        dt = torch.bfloat16 if i % 2 else torch.float16
        Hq = torch.view_as_real(torch.from_numpy(d["H"])).to(dt).contiguous()
        Yq = torch.view_as_real(torch.from_numpy(d["Y"])).to(dt).contiguous()
        Hs = Hq.float().numpy().astype(np.float64)
        Ys = Yq.float().numpy().astype(np.float64)
        refs.append((Hs[..., 0] + 1j * Hs[..., 1], Ys[..., 0] + 1j * Ys[..., 1], d["N0"]))
        cells.append(ocd.make_cell(Hq.cuda(), Yq.cuda(), d["N0"], 1.0, s["K"], s["mode"], s["order"]))
    ocd.ocd_detect_batched(cells)
    torch.cuda.synchronize()
    for s, (H, Y, N0), c in zip(specs, refs, cells):
        assert_parity(c.xhat.cpu().numpy(), c.llr.cpu().numpy(), H, Y, N0, 1.0, s["K"],
                      MODE[s["mode"]], s["order"], f"16-bit {s}")
