"""Uncoded bit error rate of the GPU detector on i.i.d. Rayleigh channels
(an i.i.d. analogue of the paper's error-rate comparison, Figs. 1-2): OCD-MMSE
and OCD-BOX for K = 1..4 sweeps against the explicit MMSE equalizer of
Eqs. 4-5 (FP64 oracle, exact mu of Section II-E) at 128x8, 64-QAM, SNR
5..30 dB.  Checks what the method guarantees: OCD-MMSE approaches the
explicit MMSE detector as K grows (it is Gauss-Seidel on the same linear
system), every detector's BER falls with SNR; the table is printed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

SNRS = [5, 10, 15, 20, 25, 30]


def mmse_bits(d, order):
    """Hard decisions of the explicit MMSE estimate: signs of the max-log
    LLRs of z / mu with the exact mu (nearest constellation point)."""
    z = orc.mmse_closed_form(d["H"], d["Y"], d["N0"], 1.0)
    mu, _ = orc.exact_mu_rho(d["H"], d["N0"], 1.0)
    n = np.sum(np.abs(np.asarray(d["H"], dtype=np.complex128)) ** 2, axis=1)
    return orc.ocd_llr(z, n, mu, d["N0"], 1.0, order) > 0


def test_uncoded_ber_against_explicit_mmse(capsys):
    order, Nsc = 64, 1500
    table = {}
    for snr in SNRS:
        d = synth.make_uplink(Nsc, 128, 8, 14, order, float(snr), 900 + snr)
        sent = d["bits"].astype(bool)
        row = {"MMSE (explicit)": float(np.mean(mmse_bits(d, order) != sent))}
        H = torch.from_numpy(d["H"]).cuda()
        Y = torch.from_numpy(d["Y"]).cuda()
        for mode in ("mmse", "box"):
            for K in (1, 2, 3, 4):
                _, L = ocd.ocd_detect(H, Y, d["N0"], 1.0, K, mode, order)
                row[f"OCD-{mode.upper()} K={K}"] = float(np.mean((L.cpu().numpy() > 0) != sent))
        table[snr] = row
    names = list(table[SNRS[0]].keys())
    with capsys.disabled():
        print("\nuncoded BER, 128x8 64-QAM, i.i.d. Rayleigh, 1500 subcarriers x 14 symbols")
        print("SNR dB " + " ".join(f"{n:>16s}" for n in names))
        for snr in SNRS:
            print(f"{snr:6d} " + " ".join(f"{table[snr][n]:16.3e}" for n in names))
    for n in names:  # every detector improves with SNR (until no errors are left)
        v = [table[s][n] for s in SNRS]
        assert all(b <= a * 1.05 + 1e-6 for a, b in zip(v, v[1:])), (n, v)
    for snr in SNRS:  # OCD-MMSE converges to the explicit MMSE detector
        ref = table[snr]["MMSE (explicit)"]
        assert abs(table[snr]["OCD-MMSE K=4"] - ref) <= 0.05 * ref + 2e-5, (snr, table[snr])
        assert table[snr]["OCD-MMSE K=4"] <= table[snr]["OCD-MMSE K=1"] * 1.01 + 1e-6
