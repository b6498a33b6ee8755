"""H and Y stored as bfloat16 / float16 complex pairs (the precision form):
the CUDA path against the FP64 oracle evaluated on the same stored values,
at the same tolerances as float32 storage."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

from .parity import assert_parity  # noqa: E402

pytestmark = pytest.mark.gpu

DT = {"bf16": torch.bfloat16, "f16": torch.float16}
MODE = {orc.MMSE: "mmse", orc.BOX: "box"}


def quantize(x, dtype):
    """complex numpy array -> (device tensor [..., 2] of dtype, stored values
    as complex128)."""
    t = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64))).to(dtype)
    back = t.float().numpy()
    return t.contiguous().cuda(), back[..., 0].astype(np.float64) + 1j * back[..., 1]


def check16(Nsc, B, U, T, K, mode, order, snr, seed, dtype, algo, Es=1.0, label=""):
    d = synth.make_uplink(Nsc, B, U, T, order, snr, seed, Es=Es)
    Hq, Hs = quantize(d["H"], DT[dtype])
    Yq, Ys = quantize(d["Y"], DT[dtype])
    x, L = ocd.ocd_detect(Hq, Yq, d["N0"], Es, K, MODE[mode], order, algo=algo)
    torch.cuda.synchronize()
    return assert_parity(x.cpu().numpy(), L.cpu().numpy(), Hs, Ys, d["N0"], Es, K, mode, order,
                         f"{label} {dtype} [{algo}]")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("algo", ["projected", "residual"])
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_128x8_64qam(mode, algo, dtype):
    check16(20, 128, 8, 14, 3, mode, 64, 15.0, 400, dtype, algo, label="128x8")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("algo", ["projected", "residual"])
@pytest.mark.parametrize("snr", [0.0, 15.0, 30.0])
def test_256x16_k4_snr(snr, algo, dtype):
    """The 256x16, K = 4 precision-form system (two user tiles)."""
    check16(8, 256, 16, 14, 4, orc.BOX, 64, snr, 410 + int(snr), dtype, algo, label="256x16")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("B,U,T,Nsc", [
    (64, 12, 14, 9), (100, 16, 5, 7), (36, 9, 17, 5), (132, 3, 33, 4), (40, 16, 1, 6),
    (34, 5, 14, 6), (33, 7, 3, 5), (64, 1, 16, 8), (512, 16, 2, 3)])
def test_ragged_shapes(B, U, T, Nsc, dtype):
    """B % 4 != 0 (no bulk copies: load-based or residual form), U between the
    tile bounds, symbol counts around the 16-symbol pass, T = 1."""
    for algo in (["projected", "residual"] if (U <= 8 or B % 4 == 0) else ["residual"]):
        check16(Nsc, B, U, T, 3, orc.MMSE, 16, 12.0, B + U + T, dtype, algo,
                label=f"{B}x{U} T{T}")


@pytest.mark.parametrize("order", [2, 4, 16, 256])
def test_alphabets_bf16(order):
    check16(6, 64, 8, 6, 3, orc.BOX, order, 20.0, 420 + order, "bf16", "projected",
            label=f"order {order}")


def test_symbol_energy_bf16():
    check16(6, 64, 16, 6, 3, orc.MMSE, 64, 12.0, 430, "bf16", "projected", Es=2.0)


def test_complex32_input_is_f16_storage():
    d = synth.make_uplink(10, 64, 8, 14, 16, 12.0, 431)
    Hc = torch.from_numpy(d["H"]).cuda().to(torch.complex32)
    Yc = torch.from_numpy(d["Y"]).cuda().to(torch.complex32)
    Hq, _ = quantize(d["H"], torch.float16)
    Yq, _ = quantize(d["Y"], torch.float16)
    x1, L1 = ocd.ocd_detect(Hc, Yc, d["N0"], 1.0, 3, "box", 16)
    x2, L2 = ocd.ocd_detect(Hq, Yq, d["N0"], 1.0, 3, "box", 16)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(L1, L2)


def test_projected_sixteen_users_needs_bulk_copy_shape():
    d = synth.make_uplink(4, 66, 16, 4, 16, 12.0, 432)  # B % 4 != 0
    Hq, _ = quantize(d["H"], torch.bfloat16)
    Yq, _ = quantize(d["Y"], torch.bfloat16)
    with pytest.raises(ocd.OcdError, match="UNSUPPORTED"):
        ocd.ocd_detect(Hq, Yq, d["N0"], 1.0, 3, "box", 16, algo="projected")
    ocd.ocd_detect(Hq, Yq, d["N0"], 1.0, 3, "box", 16)  # auto -> residual form


def test_storage_error_vs_float_inputs_is_small_at_moderate_snr():
    """Accuracy of the precision form against the FP64 oracle on the
    unquantized inputs (what 16-bit storage costs): at 15 dB the hard
    decisions agree almost everywhere."""
    d = synth.make_uplink(40, 128, 8, 14, 64, 15.0, 433, dtype=np.complex128)
    z_ref, L_ref = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 3, orc.BOX, 64)
    for dtype in ("bf16", "f16"):
        Hq, _ = quantize(d["H"], DT[dtype])
        Yq, _ = quantize(d["Y"], DT[dtype])
        x, L = ocd.ocd_detect(Hq, Yq, d["N0"], 1.0, 3, "box", 64)
        torch.cuda.synchronize()
        agree = np.mean((L.cpu().numpy() > 0) == (L_ref > 0))
        assert agree > 0.995, (dtype, agree)


def test_error_per_snr_against_the_fp64_reference(capsys):
    """The precision-form system (256x16, K = 4, 64-QAM, T = 14): per SNR
    0..30 dB, the error of each storage against the FP64 oracle on the
    unquantized inputs (what 16-bit storage costs), printed as a table."""
    import math
    rows = []
    for snr in range(0, 31, 5):
        d = synth.make_uplink(48, 256, 16, 14, 64, float(snr), 100 + snr, dtype=np.complex128)
        z_ref, l_ref = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 4, orc.BOX, 64)
        for name, dt in (("f32", None), ("bf16", torch.bfloat16), ("f16", torch.float16)):
            if dt is None:
                H = torch.from_numpy(d["H"].astype(np.complex64)).cuda()
                Y = torch.from_numpy(d["Y"].astype(np.complex64)).cuda()
            else:
                H, _ = quantize(d["H"], dt)
                Y, _ = quantize(d["Y"], dt)
            x, L = ocd.ocd_detect(H, Y, d["N0"], 1.0, 4, "box", 64)
            torch.cuda.synchronize()
            x = x.cpu().numpy()
            L = L.cpu().numpy()
            xe = float(np.max(np.linalg.norm(x - z_ref, axis=-1)
                              / np.maximum(np.linalg.norm(z_ref, axis=-1), 1e-3 * math.sqrt(16))))
            le = float(np.quantile(np.abs(L - l_ref) / np.maximum(np.abs(l_ref), 1.0), 0.99))
            mm = float(np.mean((L > 0) != (l_ref > 0)))
            rows.append((snr, name, xe, le, mm))
            bound = {"f32": (1e-4, 1e-3, 1e-3), "bf16": (1e-2, 5e-2, 5e-3),
                     "f16": (2e-3, 1e-2, 1e-3)}[name]
            assert xe <= bound[0] and le <= bound[1] and mm <= bound[2], (snr, name, xe, le, mm)
    with capsys.disabled():
        print("\nSNR dB  storage  xhat rel err max  LLR rel err p99  hard-bit mismatch")
        for snr, name, xe, le, mm in rows:
            print(f"{snr:6d}  {name:7s}  {xe:16.2e}  {le:15.2e}  {mm:17.2e}")
