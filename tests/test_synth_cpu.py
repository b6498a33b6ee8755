"""The seeded input recipe (the synthetic stand-in for the paper's LTE-A /
WINNER-II workload): channel statistics, noise level, bit mapping, the
mixed-cell parameters of the batched workload, and determinism."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1611_08779_gb300 import synth


def test_channel_columns_have_unit_energy_on_average():
    """H i.i.d. CN(0, 1/B): E ||h_u||^2 = 1 and real/imaginary parts each of
    variance 1/(2B), independent of each other."""
    d = synth.make_uplink(400, 64, 8, 1, 16, 10.0, seed=31, dtype=np.complex128)
    H = d["H"]
    n = np.sum(np.abs(H) ** 2, axis=1)  # [Nsc, U]
    assert abs(n.mean() - 1.0) < 0.01
    assert abs(H.real.var() - 1 / 128) < 2e-4 and abs(H.imag.var() - 1 / 128) < 2e-4
    assert abs(np.mean(H.real * H.imag)) < 2e-4


@pytest.mark.parametrize("snr_db", [0.0, 15.0, 30.0])
def test_noise_variance_follows_the_snr_reading(snr_db):
    """N0 = Es 10^(-SNR/10) and Y - H S is CN(0, N0) per entry."""
    d = synth.make_uplink(300, 32, 4, 7, 64, snr_db, seed=32, dtype=np.complex128)
    assert math.isclose(d["N0"], 10 ** (-snr_db / 10), rel_tol=1e-12)
    N = d["Y"] - np.matmul(d["S"], np.swapaxes(d["H"], 1, 2))
    assert abs(np.mean(np.abs(N) ** 2) / d["N0"] - 1.0) < 0.02


@pytest.mark.parametrize("order", [2, 4, 16, 64, 256])
def test_symbols_are_the_mapped_bits_with_unit_energy(order):
    d = synth.make_uplink(200, 16, 4, 14, order, 20.0, seed=33, dtype=np.complex128)
    assert np.array_equal(d["S"], synth.map_bits(d["bits"], order))
    pts, _ = orc.alphabet(order)
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-12
    assert abs(np.mean(np.abs(d["S"]) ** 2) - 1.0) < 0.03
    # every transmitted symbol is a point of the alphabet
    dist = np.min(np.abs(d["S"].reshape(-1, 1) - pts[None, :]), axis=1)
    assert np.max(dist) < 1e-12


def test_symbol_energy_scales_the_alphabet():
    d = synth.make_uplink(50, 8, 2, 3, 16, 10.0, seed=34, Es=2.5, dtype=np.complex128)
    pts, _ = orc.alphabet(16, 2.5)
    dist = np.min(np.abs(d["S"].reshape(-1, 1) - pts[None, :]), axis=1)
    assert np.max(dist) < 1e-12
    assert math.isclose(d["N0"], 2.5 * 10 ** (-1.0), rel_tol=1e-12)


def test_draws_are_seeded_and_stored_in_the_requested_type():
    a = synth.make_uplink(5, 8, 2, 3, 16, 10.0, seed=35)
    b = synth.make_uplink(5, 8, 2, 3, 16, 10.0, seed=35)
    c = synth.make_uplink(5, 8, 2, 3, 16, 10.0, seed=36)
    assert a["H"].dtype == np.complex64 and a["Y"].dtype == np.complex64
    assert np.array_equal(a["H"], b["H"]) and np.array_equal(a["Y"], b["Y"])
    assert not np.array_equal(a["H"], c["H"])
    assert a["H"].flags.c_contiguous and a["Y"].flags.c_contiguous
    assert a["H"].shape == (5, 8, 2) and a["Y"].shape == (5, 3, 8)


def test_mixed_cells_follow_the_batched_recipe():
    specs = synth.mixed_cell_specs(24, seed=12)
    assert len(specs) == 24
    pairs = [(32, 4), (64, 8), (128, 16), (256, 32)]
    for i, s in enumerate(specs):
        assert (s["B"], s["U"]) == pairs[i % 4]
        assert s["T"] == (1, 7, 14)[(i // 4) % 3]
        assert 300 <= s["Nsc"] <= 3300 and 2 <= s["K"] <= 5
        assert s["mode"] in ("box", "mmse") and s["order"] in (16, 64)
        assert 5.0 <= s["snr_db"] <= 25.0
    # every (B, U) pair meets every symbol count
    assert {(s["B"], s["T"]) for s in specs} == {(b, t) for b, _ in pairs for t in (1, 7, 14)}
    assert synth.mixed_cell_specs(24, seed=12) == specs
