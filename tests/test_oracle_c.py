"""The plain-C FP64 oracle (oracle/ocd_ref.c) against the NumPy oracle and the
closed forms that pin it.

The C oracle exists so that the CPU baseline runs on every host core; it is
trusted only as far as these checks go: agreement with the pinned NumPy
oracle to rounding order on every mode, alphabet and edge case, plus two
closed forms checked on the C side directly (MMSE convergence, Eqs. 4-5;
noiseless recovery at B >> U), and thread-count independence.
"""
import shutil

import numpy as np
import pytest

import oracle as orc
from paper_1611_08779_gb300 import synth

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")


@pytest.fixture(scope="module")
def native():
    from oracle import native as nat
    nat.build()
    return nat


def _xerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _lerr(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))


CASES = [
    # (Nsc, B, U, T, K, order, snr)
    (5, 32, 8, 1, 3, 16, 10.0),
    (3, 128, 8, 14, 3, 64, 15.0),
    (4, 16, 4, 3, 5, 4, 0.0),
    (2, 64, 16, 2, 4, 256, 30.0),
    (3, 8, 2, 5, 2, 2, 5.0),
    (2, 33, 7, 3, 6, 64, 20.0),   # odd sizes
    (1, 256, 32, 1, 2, 16, 12.0),  # largest user count
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_c_oracle_matches_numpy_oracle(native, case, mode):
    Nsc, B, U, T, K, order, snr = case
    d = synth.make_uplink(Nsc, B, U, T, order, snr, seed=100 + CASES.index(case), dtype=np.complex128)
    z_ref, L_ref = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, K, mode, order)
    z, L = native.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, K, mode, order)
    # same steps in another summation order: relative differences of a few ulps,
    # amplified in the LLR only by rho (<= ~1e3 here)
    assert _xerr(z, z_ref) < 1e-12
    assert _lerr(L, L_ref) < 1e-10
    assert np.array_equal(orc.hard_bits(L), orc.hard_bits(L_ref))


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_c_oracle_general_es_and_zero_column(native, mode):
    d = synth.make_uplink(3, 16, 4, 2, 16, 8.0, seed=11, Es=2.5, dtype=np.complex128)
    H = d["H"].copy()
    H[:, :, 2] = 0.0          # zero column: z_u stays 0, its LLRs are 0
    z_ref, L_ref = orc.ocd_detect(H, d["Y"], d["N0"], 2.5, 4, mode, 16)
    z, L = native.ocd_detect(H, d["Y"], d["N0"], 2.5, 4, mode, 16)
    assert np.all(z[:, :, 2] == 0) and np.all(L[:, :, 2] == 0)
    assert _xerr(z, z_ref) < 1e-12
    assert _lerr(L, L_ref) < 1e-10


def test_c_oracle_zero_sweeps_and_no_llr(native):
    d = synth.make_uplink(2, 8, 3, 2, 64, 10.0, seed=12, dtype=np.complex128)
    z, L = native.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 0, orc.BOX, 64, want_llr=False)
    assert L is None and np.all(z == 0)
    z, _ = native.ocd_detect(d["H"], d["Y"], 0.0, 1.0, 3, orc.BOX, 64, want_llr=False)
    z_ref, _ = orc.ocd_detect(d["H"], d["Y"], 0.0, 1.0, 3, orc.BOX, 64, want_llr=False)
    assert _xerr(z, z_ref) < 1e-12


def test_c_oracle_rejects_bad_arguments(native):
    d = synth.make_uplink(1, 8, 2, 1, 16, 10.0, seed=13, dtype=np.complex128)
    with pytest.raises(ValueError):
        native.ocd_detect(d["H"], d["Y"], 0.0, 1.0, 3, orc.BOX, 16)  # LLRs need N0 > 0
    with pytest.raises(ValueError):
        native.ocd_detect(d["H"], d["Y"], 0.1, 0.0, 3, orc.BOX, 16)  # Es must be > 0


def test_c_oracle_mmse_converges_to_closed_form(native):
    """Eqs. 4-5 on the C side: Gauss-Seidel on the SPD system converges."""
    d = synth.make_uplink(4, 32, 8, 2, 16, 10.0, 4, dtype=np.complex128)
    H, Y, N0 = d["H"], d["Y"], d["N0"]
    G = np.conj(np.swapaxes(H, 1, 2)) @ H + N0 * np.eye(8)
    ref = np.linalg.solve(G, np.conj(np.swapaxes(H, 1, 2)) @ np.swapaxes(Y, 1, 2))
    ref = np.swapaxes(ref, 1, 2)
    z, _ = native.ocd_detect(H, Y, N0, 1.0, 200, orc.MMSE, 16, want_llr=False)
    assert _xerr(z, ref) < 1e-10


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_c_oracle_noiseless_recovery(native, mode):
    d = synth.make_noiseless(4, 128, 8, 3, 64, seed=7)
    z, L = native.ocd_detect(d["H"], d["Y"], 1e-12, 1.0, 60, mode, 64)
    assert np.max(np.abs(z - d["S"])) < 1e-6
    assert np.array_equal(orc.hard_bits(L), d["bits"])


def test_c_oracle_thread_count_does_not_change_results(native):
    d = synth.make_uplink(40, 32, 4, 3, 16, 10.0, seed=14, dtype=np.complex128)
    z1, L1 = native.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 3, orc.BOX, 16, threads=1)
    z4, L4 = native.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 3, orc.BOX, 16, threads=4)
    assert np.array_equal(z1, z4) and np.array_equal(L1, L4)
    assert native.max_threads() >= 1
