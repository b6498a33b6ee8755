"""GPU parity of the one-symbol projected form (T = 1, U <= 8, float32
storage, even B, aligned H and Y: one lane per subcarrier) against the FP64
oracle, through the C ABI.

Covers every user count of the kernel table (1..8), both modes, all
alphabets, antenna counts that leave a short last step (B not a multiple of
the antennas per step), ragged groups of 32 subcarriers, K = 0 and large K,
a zero column, Es != 1, and the full 128x8 T = 1 workload (several groups
per warp) on sampled subcarriers.  Tolerances in tests/parity.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

from .parity import assert_parity  # noqa: E402

pytestmark = pytest.mark.gpu

MODE = {orc.MMSE: "mmse", orc.BOX: "box"}


def run(d, K, mode, order, Es=1.0, algo="auto", H=None):
    Hh = d["H"] if H is None else H
    x, L = ocd.ocd_detect(torch.from_numpy(Hh).cuda(), torch.from_numpy(d["Y"]).cuda(),
                          d["N0"], Es, K, MODE[mode], order, algo=algo)
    torch.cuda.synchronize()
    return x.cpu().numpy(), L.cpu().numpy()


def check(Nsc, B, U, K, mode, order, snr, seed, Es=1.0, algo="auto"):
    d = synth.make_uplink(Nsc, B, U, 1, order, snr, seed, Es=Es)
    x, L = run(d, K, mode, order, Es, algo)
    assert_parity(x, L, d["H"], d["Y"], d["N0"], Es, K, mode, order,
                  f"lane {B}x{U} Nsc={Nsc} K={K} {MODE[mode]} {order}-QAM [{algo}]")


@pytest.mark.parametrize("U", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_every_user_count(mode, U):
    check(75, 34, U, 3, mode, 16, 12.0, 300 + U)


@pytest.mark.parametrize("B", [2, 4, 6, 18, 30, 128, 130, 256, 510, 512])
@pytest.mark.parametrize("U", [1, 3, 8])
def test_antenna_counts_and_short_last_step(B, U):
    check(40, B, U, 3, orc.BOX, 64, 15.0, 400 + B + U)


@pytest.mark.parametrize("Nsc", [1, 31, 32, 33, 64, 95, 1000])
def test_ragged_groups(Nsc):
    check(Nsc, 64, 8, 3, orc.MMSE, 64, 10.0, 500 + Nsc)


@pytest.mark.parametrize("order", [2, 4, 16, 64, 256])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_every_alphabet(mode, order):
    check(50, 32, 8, 3, mode, order, 20.0, 600 + order)


@pytest.mark.parametrize("K", [0, 1, 2, 8, 40])
def test_sweep_counts(K):
    check(40, 32, 6, K, orc.BOX, 16, 8.0, 700 + K)


def test_symbol_energy_not_one():
    check(40, 32, 8, 4, orc.MMSE, 64, 18.0, 800, Es=2.5)
    check(40, 32, 8, 4, orc.BOX, 64, 18.0, 801, Es=2.5)


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_zero_column(mode):
    d = synth.make_uplink(40, 32, 8, 1, 16, 10.0, 900)
    H = d["H"].copy()
    H[:, :, 5] = 0
    x, L = run(d, 3, mode, 16, H=H)
    assert np.all(x[:, :, 5] == 0) and np.all(L[:, :, 5] == 0)
    assert_parity(x, L, H, d["Y"], d["N0"], 1.0, 3, mode, 16, "lane zero column")


def test_projected_and_auto_agree_bitwise():
    """AUTO picks the same kernel as an explicit PROJECTED request at T = 1."""
    d = synth.make_uplink(200, 128, 8, 1, 64, 15.0, 901)
    xa, La = run(d, 3, orc.BOX, 64, algo="auto")
    xp, Lp = run(d, 3, orc.BOX, 64, algo="projected")
    assert np.array_equal(xa, xp) and np.array_equal(La, Lp)


def test_full_128x8_workload_sampled():
    """80,000 subcarriers (2500 groups: more than one per warp): sampled subcarriers
    against the oracle, every output finite."""
    Nsc = 80000
    d = synth.make_uplink(Nsc, 128, 8, 1, 64, 15.0, 902)
    x, L = run(d, 3, orc.BOX, 64)
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(L))
    rng = np.random.default_rng(903)
    idx = np.unique(np.concatenate([rng.integers(0, Nsc, 300), [0, 31, 32, Nsc - 33, Nsc - 1]]))
    assert_parity(x[idx], L[idx], d["H"][idx], d["Y"][idx], d["N0"], 1.0, 3, orc.BOX, 64,
                  "lane 128x8 full workload (sampled)")
