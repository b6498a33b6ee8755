"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.  Tolerances in tests/parity.py."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

from .parity import assert_parity, xhat_error  # noqa: E402

pytestmark = pytest.mark.gpu

MODE = {orc.MMSE: "mmse", orc.BOX: "box"}
ALGOS = ["residual", "projected"]


def algos_for(U, B=None):
    """Arrangements supporting the shape: projected for U <= 8, and for
    U <= 32 when B is even (the bulk-copy kernels; test arrays are aligned)."""
    if U <= 8 or (U <= 32 and B is not None and B % 2 == 0):
        return ALGOS
    return ["residual"]


def run_gpu(d, K, mode, order, Es=1.0, N0=None, want_xhat=True, want_llr=True, algo="auto"):
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    x, L = ocd.ocd_detect(H, Y, d["N0"] if N0 is None else N0, Es, K, MODE[mode], order,
                          want_xhat=want_xhat, want_llr=want_llr, algo=algo)
    torch.cuda.synchronize()
    return (x.cpu().numpy() if x is not None else None,
            L.cpu().numpy() if L is not None else None)


def check(Nsc, B, U, T, K, mode, order, snr, seed, Es=1.0, label="", algos=None):
    """Every arrangement that supports the shape must match the oracle."""
    d = synth.make_uplink(Nsc, B, U, T, order, snr, seed, Es=Es)
    out = {}
    for algo in (algos or algos_for(U, B)):
        x, L = run_gpu(d, K, mode, order, Es, algo=algo)
        out[algo] = assert_parity(x, L, d["H"], d["Y"], d["N0"], Es, K, mode, order,
                                  f"{label} [{algo}]")
    return out


# Small configuration of the paper's 32x8 system: 64 subcarriers, T = 1, K = 3,
# 16-QAM at 10 dB, OCD-MMSE.
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_32x8_16qam_t1(mode):
    check(64, 32, 8, 1, 3, mode, 16, 10.0, 0, label="32x8")


# The 128x8 64-QAM K=3 T=14 system over the SNR sweep (a slice of subcarriers).
@pytest.mark.parametrize("snr", [0.0, 10.0, 20.0, 30.0])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_128x8_64qam_t14_snr_sweep(mode, snr):
    check(24, 128, 8, 14, 3, mode, 64, snr, int(snr) + 1, label=f"128x8 {snr}dB")


@pytest.mark.parametrize("order", [2, 4, 16, 64, 256])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_every_alphabet(mode, order):
    check(9, 64, 6, 5, 4, mode, order, 18.0, 3, label=f"order {order}")


# Ragged shapes: odd B (scalar Y loads, padded antennas), U not a power of
# two, T not dividing the CTA chunk, many chunks with a partial last one.
@pytest.mark.parametrize("B,U,T,Nsc", [
    (37, 5, 3, 29), (1, 1, 1, 5), (3, 2, 7, 11), (4, 8, 2, 6), (130, 7, 13, 17),
    (200, 12, 9, 10), (96, 16, 14, 8), (64, 32, 3, 5), (256, 16, 14, 6),
    (512, 32, 2, 3), (512, 1, 5, 4), (33, 17, 1, 40), (17, 3, 33, 3)])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_ragged_shapes(mode, B, U, T, Nsc):
    check(Nsc, B, U, T, 3, mode, 16, 12.0, B * 7 + U, label=f"{B}x{U} T{T}")


@pytest.mark.parametrize("K", [0, 1, 2, 5, 16])
def test_sweep_counts(K):
    check(10, 48, 6, 4, K, orc.MMSE, 64, 15.0, 40 + K, label=f"K={K}")
    check(10, 48, 6, 4, K, orc.BOX, 64, 5.0, 50 + K, label=f"K={K}")


def test_maximum_sweeps_box():
    check(3, 16, 4, 2, 256, orc.BOX, 16, 5.0, 60, label="K=256")


def test_symbol_energy_not_one():
    check(8, 64, 8, 6, 3, orc.MMSE, 64, 12.0, 61, Es=2.5)
    check(8, 64, 8, 6, 3, orc.BOX, 16, 12.0, 62, Es=0.3)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_zero_column(mode, algo):
    d = synth.make_uplink(6, 32, 5, 3, 16, 10.0, 63)
    d["H"][:, :, 3] = 0
    d["H"][2, :, 0] = 0
    x, L = run_gpu(d, 3, mode, 16, algo=algo)
    assert np.all(x[:, :, 3] == 0) and np.all(L[:, :, 3] == 0)
    assert_parity(x, L, d["H"], d["Y"], d["N0"], 1.0, 3, mode, 16)


@pytest.mark.parametrize("algo", ALGOS)
def test_least_squares_mmse_with_zero_noise(algo):
    d = synth.make_uplink(5, 64, 8, 3, 64, 20.0, 64)
    x, L = run_gpu(d, 6, orc.MMSE, 64, N0=0.0, want_llr=False, algo=algo)
    assert L is None
    z_ref, *_ = orc.ocd_equalize(d["H"], d["Y"], 0.0, 1.0, 6, orc.MMSE, 64)
    assert xhat_error(x, z_ref) <= 1e-4


@pytest.mark.parametrize("algo", ALGOS)
def test_outputs_optional(algo):
    d = synth.make_uplink(5, 32, 4, 3, 16, 10.0, 65)
    x1, L1 = run_gpu(d, 3, orc.BOX, 16, algo=algo)
    x2, L2 = run_gpu(d, 3, orc.BOX, 16, want_llr=False, algo=algo)
    x3, L3 = run_gpu(d, 3, orc.BOX, 16, want_xhat=False, algo=algo)
    assert L2 is None and x3 is None
    assert np.array_equal(x1, x2) and np.array_equal(L1, L3)


def test_empty_inputs():
    H = torch.zeros((0, 16, 4), dtype=torch.complex64, device="cuda")
    Y = torch.zeros((0, 3, 16), dtype=torch.complex64, device="cuda")
    x, L = ocd.ocd_detect(H, Y, 0.1, qam_order=16)
    assert x.shape == (0, 3, 4) and L.shape == (0, 3, 4, 4)
    H = torch.zeros((4, 16, 4), dtype=torch.complex64, device="cuda")
    Y = torch.zeros((4, 0, 16), dtype=torch.complex64, device="cuda")
    x, L = ocd.ocd_detect(H, Y, 0.1, qam_order=16)
    torch.cuda.synchronize()
    assert x.shape == (4, 0, 4)


@pytest.mark.parametrize("algo", ALGOS)
def test_noiseless_recovery_on_gpu(algo):
    d = synth.make_noiseless(16, 128, 8, 14, 64, seed=66)
    d["H"] = d["H"].astype(np.complex64)
    d["Y"] = d["Y"].astype(np.complex64)
    d["N0"] = 1e-6
    x, L = run_gpu(d, 8, orc.BOX, 64, algo=algo)
    assert np.array_equal((L > 0).astype(np.uint8), d["bits"])


@pytest.mark.parametrize("algo", ALGOS)
def test_deterministic_and_stream_independent(algo):
    d = synth.make_uplink(40, 128, 8, 14, 64, 15.0, 67)
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    x1, L1 = ocd.ocd_detect(H, Y, d["N0"], 1.0, 3, "box", 64, algo=algo)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        x2, L2 = ocd.ocd_detect(H, Y, d["N0"], 1.0, 3, "box", 64, algo=algo)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(L1, L2)


@pytest.mark.parametrize("algo", ALGOS)
def test_unaligned_y_uses_scalar_loads(algo):
    # Y starting 8 bytes past a 16-byte boundary takes the scalar-load path
    d = synth.make_uplink(6, 64, 8, 3, 16, 10.0, 68)
    H = torch.from_numpy(d["H"]).cuda()
    flat = torch.zeros(d["Y"].size + 1, dtype=torch.complex64, device="cuda")
    flat[1:] = torch.from_numpy(d["Y"].reshape(-1)).cuda()
    Y = flat[1:].view(d["Y"].shape)
    assert Y.data_ptr() % 16 == 8
    x, L = ocd.ocd_detect(H, Y, d["N0"], 1.0, 3, "mmse", 16, algo=algo)
    torch.cuda.synchronize()
    assert_parity(x.cpu().numpy(), L.cpu().numpy(), d["H"], d["Y"], d["N0"], 1.0, 3,
                  orc.MMSE, 16)


def test_host_entry_point_matches_device_entry_point():
    d = synth.make_uplink(50, 128, 8, 14, 64, 12.0, 69)
    Hh = torch.from_numpy(d["H"]).pin_memory()
    Yh = torch.from_numpy(d["Y"]).pin_memory()
    xh, Lh = ocd.ocd_detect_host(Hh, Yh, d["N0"], 1.0, 3, "box", 64, pieces=3)
    xd, Ld = ocd.ocd_detect(Hh.cuda(), Yh.cuda(), d["N0"], 1.0, 3, "box", 64)
    torch.cuda.synchronize()
    assert torch.equal(xh, xd.cpu()) and torch.equal(Lh, Ld.cpu())


@pytest.mark.parametrize("algo", ["auto", "residual", "projected"])
def test_full_size_sampled_against_oracle(algo):
    """128x8, 64-QAM, K = 3, T = 14 over 1200 x 4 subcarriers in one launch,
    as the benchmark launches it; sampled subcarriers go to the oracle."""
    Nsc = 1200 * 4
    d = synth.make_uplink(Nsc, 128, 8, 14, 64, 15.0, 70)
    x, L = run_gpu(d, 3, orc.BOX, 64, algo=algo)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(Nsc, 48, replace=False))
    idx[0], idx[-1] = 0, Nsc - 1
    assert_parity(x[idx], L[idx], d["H"][idx], d["Y"][idx], d["N0"], 1.0, 3, orc.BOX, 64)
    assert np.all(np.isfinite(L))


@pytest.mark.parametrize("B,U", [(33, 9), (33, 17), (31, 16), (35, 32)])
def test_projected_rejects_unsupported_shapes(B, U):
    """More than 8 users with odd B (no bulk-copy staging)."""
    d = synth.make_uplink(2, B, U, 2, 16, 10.0, 71)
    with pytest.raises(ocd.OcdError, match="UNSUPPORTED"):
        run_gpu(d, 3, orc.MMSE, 16, algo="projected")
    x, L = run_gpu(d, 3, orc.MMSE, 16, algo="auto")  # falls back to the residual form
    assert_parity(x, L, d["H"], d["Y"], d["N0"], 1.0, 3, orc.MMSE, 16)


@pytest.mark.parametrize("U", [9, 12, 16])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_projected_two_user_tiles(mode, U):
    """9..16 users (two 8-user MMA tiles) in float32 storage, several passes."""
    check(7, 96, U, 20, 4, mode, 64, 18.0, 500 + U, label=f"96x{U}", algos=["projected"])


@pytest.mark.parametrize("T", [1, 2, 15, 16, 17, 33, 40])
@pytest.mark.parametrize("U", [1, 3, 4, 5, 8])
def test_projected_symbol_passes_and_user_bounds(U, T):
    """Symbol counts around the per-pass width (16 symbols for U <= 8, 32 for
    U <= 4) and user counts around both instance bounds."""
    check(5, 40, U, T, 3, orc.BOX, 16, 8.0, 100 * U + T, label=f"U{U} T{T}",
          algos=["projected"])


@pytest.mark.parametrize("U", [17, 20, 24, 31, 32])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_projected_four_user_tiles(mode, U):
    """17..32 users (four 8-user tiles, G phase then q0 passes) in float32
    storage: ragged last antenna block, several symbol passes."""
    check(5, 100, U, 20, 4, mode, 64, 18.0, 600 + U, label=f"100x{U}", algos=["projected"])


@pytest.mark.parametrize("T", [1, 2, 5, 7, 8, 9])
@pytest.mark.parametrize("B,U", [(34, 17), (130, 32), (2, 24)])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_projected_wide_up_to_eight_symbols(mode, B, U, T):
    """17..32 users with T <= 8 (q0 accumulated in the G phase, no q0 pass)
    and T = 9 (one q0 pass), ragged antenna blocks."""
    check(7, B, U, T, 3, mode, 64, 16.0, 700 + B + U + T, label=f"{B}x{U} T{T}",
          algos=["projected"])


@pytest.mark.parametrize("B,U,T", [(256, 32, 14), (256, 32, 1), (512, 32, 2), (34, 18, 17),
                                   (64, 32, 16), (2, 17, 3)])
def test_projected_wide_shapes(B, U, T):
    """The 256x32 cells of the batched workload, B = 512, tiny B, T = 1."""
    check(4, B, U, T, 3, orc.BOX, 16, 15.0, B + U + T, label=f"{B}x{U} T{T}",
          algos=["projected"])


@pytest.mark.parametrize("order", [4, 16, 64, 256])
@pytest.mark.parametrize("U", [8, 16])
def test_llr_array_only_4_byte_aligned(U, order):
    """An LLR array that starts 4 bytes past an 8-byte boundary takes the
    kernels' scalar store path (the paired float2 stores need 8-byte
    alignment); both paths must give the oracle's values."""
    d = synth.make_uplink(20, 64, U, 14, order, 15.0, 66 + U + order)
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    Q = orc.bits_per_symbol(order)
    n = 20 * 14 * U * Q
    for mode in (orc.MMSE, orc.BOX):
        buf = torch.full((n + 1,), float("nan"), dtype=torch.float32, device="cuda")
        llr = buf[1:].view(20, 14, U, Q)
        assert llr.data_ptr() % 8 == 4
        x, L = ocd.ocd_detect(H, Y, d["N0"], 1.0, 3, MODE[mode], order, llr=llr, algo="projected")
        torch.cuda.synchronize()
        assert L.data_ptr() == llr.data_ptr()
        assert_parity(x.cpu().numpy(), L.cpu().numpy(), d["H"], d["Y"], d["N0"], 1.0, 3, mode,
                      order, f"unaligned LLR U={U} order={order}")
        assert bool(torch.isnan(buf[0]))  # the slot before the array is untouched
