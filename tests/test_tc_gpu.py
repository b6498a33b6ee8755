"""The tcgen05 (tensor-memory) kernel of the projected form, 16 < U <= 32 and
T <= 16: element-wise parity with the FP64 oracle over ragged antenna
blocks, user counts that are not multiples of 8, symbol counts on both sides
of the 8-row received-vector box, subcarrier counts from one to several per
CTA; agreement with the warp-level MMA kernel; determinism; the fallback
beyond 16 symbols; sampled parity at the 256x32 benchmark size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

from .parity import assert_parity, xhat_error  # noqa: E402

pytestmark = pytest.mark.gpu
MODE = {orc.MMSE: "mmse", orc.BOX: "box"}


def run(d, K, mode, order, algo, Es=1.0):
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    x, L = ocd.ocd_detect(H, Y, d["N0"], Es, K, MODE[mode], order, algo=algo)
    torch.cuda.synchronize()
    return x.cpu().numpy(), L.cpu().numpy()


@pytest.mark.parametrize("B,U,T,Nsc", [
    (64, 32, 14, 7), (256, 32, 14, 5), (128, 17, 1, 9), (130, 24, 7, 11), (18, 31, 8, 6),
    (2, 20, 9, 4), (512, 32, 16, 3), (66, 25, 3, 300), (256, 32, 1, 160), (34, 32, 13, 1)])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_parity_with_the_oracle(mode, B, U, T, Nsc):
    d = synth.make_uplink(Nsc, B, U, T, 64, 14.0, B + 3 * U + T)
    x, L = run(d, 3, mode, 64, "projected_tc")
    assert_parity(x, L, d["H"], d["Y"], d["N0"], 1.0, 3, mode, 64, f"tc {B}x{U} T{T}")
    assert ocd.fault_status(clear=False) == 0


@pytest.mark.parametrize("order", [2, 4, 16, 256])
@pytest.mark.parametrize("K", [0, 1, 5])
def test_alphabets_and_sweep_counts(order, K):
    d = synth.make_uplink(12, 96, 28, 10, order, 20.0, 70 + order + K)
    for mode in (orc.MMSE, orc.BOX):
        x, L = run(d, K, mode, order, "projected_tc")
        assert_parity(x, L, d["H"], d["Y"], d["N0"], 1.0, K, mode, order, f"order {order} K={K}")


def test_symbol_energy_and_zero_columns():
    d = synth.make_uplink(10, 64, 24, 14, 16, 12.0, 81, Es=2.5)
    d["H"][:, :, 5] = 0
    d["H"][3, :, 20] = 0
    for mode in (orc.MMSE, orc.BOX):
        x, L = run(d, 3, mode, 16, "projected_tc", Es=2.5)
        assert np.all(x[:, :, 5] == 0) and np.all(L[:, :, 5] == 0)
        assert_parity(x, L, d["H"], d["Y"], d["N0"], 2.5, 3, mode, 16, "Es=2.5, zero columns")


@pytest.mark.parametrize("T", [1, 8, 14, 16])
def test_agrees_with_the_warp_level_kernel(T):
    d = synth.make_uplink(40, 128, 32, T, 64, 18.0, 90 + T)
    x1, L1 = run(d, 4, orc.BOX, 64, "projected_tc")
    x2, L2 = run(d, 4, orc.BOX, 64, "projected_warp")
    assert xhat_error(x1, x2) <= 2e-5
    assert np.max(np.abs(L1 - L2) / np.maximum(np.abs(L2), 1.0)) <= 1e-3


def test_deterministic():
    d = synth.make_uplink(500, 64, 32, 14, 16, 10.0, 95)
    r1 = run(d, 3, orc.MMSE, 16, "projected_tc")
    r2 = run(d, 3, orc.MMSE, 16, "projected_tc")
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


def test_more_than_16_symbols():
    """T = 17: the default projected form takes the warp-level kernel; an
    explicit request of the tensor-memory kernel is refused before any work."""
    d = synth.make_uplink(6, 64, 32, 17, 16, 12.0, 96)
    x, L = run(d, 3, orc.BOX, 16, "projected")
    assert_parity(x, L, d["H"], d["Y"], d["N0"], 1.0, 3, orc.BOX, 16, "T=17")
    with pytest.raises(ocd.OcdError, match="UNSUPPORTED"):
        run(d, 3, orc.BOX, 16, "projected_tc")


def test_default_projected_form_matches_the_oracle_on_both_sides_of_the_switch():
    """The library's own choice (tensor-memory kernel up to 16 symbols,
    warp-level kernel above) at T = 1, 8, 16 and 17."""
    for T in (1, 8, 16, 17):
        d = synth.make_uplink(30, 128, 32, T, 64, 16.0, 98 + T)
        x, L = run(d, 3, orc.MMSE, 64, "projected")
        assert_parity(x, L, d["H"], d["Y"], d["N0"], 1.0, 3, orc.MMSE, 64, f"T={T}")


def test_benchmark_size_sampled():
    """256x32, T = 14, K = 4, 64-QAM, 4000 subcarriers in one launch (about
    26 subcarriers per CTA, every TMEM slot reused); every 37th subcarrier
    against the oracle."""
    d = synth.make_uplink(4000, 256, 32, 14, 64, 15.0, 97)
    x, L = run(d, 4, orc.BOX, 64, "projected_tc")
    idx = np.arange(0, 4000, 37)
    assert_parity(x[idx], L[idx], d["H"][idx], d["Y"][idx], d["N0"], 1.0, 4, orc.BOX, 64,
                  "256x32 sampled")
    assert ocd.fault_status(clear=False) == 0
