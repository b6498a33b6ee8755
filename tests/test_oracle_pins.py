"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an invariant, an equivalence claimed by the paper, a hand-derived value
(tests/golden/hand_examples.json) or a brute-force solution of the same
problem.  A plausible slip in the oracle (dropped p_u z_u term, wrong sign of
the residual update, missing conjugate, wrong regularizer, swapped LLR sign or
bit order, wrong box radius) fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_1611_08779_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")
ORDERS = (2, 4, 16, 64, 256)


def _expr(v):
    if isinstance(v, str):
        return float(eval(v, {"sqrt": math.sqrt}))  # hand-written constants only
    return float(v)


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Constellation (Section II-A) and box radius (Section II-D)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("order", ORDERS)
def test_alphabet_unit_energy_gray_and_labels(order):
    pts, lab = orc.alphabet(order)
    Q = orc.bits_per_symbol(order)
    assert len(pts) == order and lab.shape == (order, Q)
    assert abs(np.mean(np.abs(pts) ** 2) - 1.0) < 1e-14          # E|s|^2 = 1
    words = {tuple(r) for r in lab}
    assert len(words) == order                                     # labels unique
    # Gray: nearest neighbours differ in exactly one bit
    d = np.abs(pts[:, None] - pts[None, :])
    dmin = np.min(d[d > 0])
    for i, j in zip(*np.nonzero(np.isclose(d, dmin))):
        assert np.sum(lab[i] != lab[j]) == 1


@pytest.mark.parametrize("order", ORDERS)
def test_box_radius_matches_hand_values(order, golden):
    assert abs(orc.box_radius(order) - _expr(golden["radius"][str(order)])) < 1e-15
    assert abs(orc.box_radius(order, Es=4.0) - 2 * _expr(golden["radius"][str(order)])) < 1e-14


@pytest.mark.parametrize("order", ORDERS)
def test_generator_mapping_agrees_with_oracle_labels(order):
    """Two independent codings of the same Gray convention (the generator
    decodes Gray words, the oracle encodes level indices) must agree."""
    pts, lab = orc.alphabet(order)
    mapped = synth.map_bits(lab, order)
    assert np.max(np.abs(mapped - pts)) < 1e-14


# --------------------------------------------------------------------------
# Hand-derived examples
# --------------------------------------------------------------------------

def test_hand_llr_16qam(golden):
    g = golden["llr_16qam"]
    z = np.array([[[complex(g["z_re_times_sqrt10"], g["z_im_times_sqrt10"]) / math.sqrt(10)]]])
    n = np.array([[g["n"]]])
    p = np.array([[g["p"]]])
    L = orc.ocd_llr(z, n, p, g["N0"], g["Es"], 16)[0, 0, 0]
    assert np.max(np.abs(L - np.array(g["llr"]))) < 1e-12


def _ortho(golden):
    g = golden["orthogonal_2x2"]
    H = (np.array(g["H_re"]) + 1j * np.array(g["H_im"]))[None]
    y = (np.array(g["y_re"]) + 1j * np.array(g["y_im"]))[None, None]
    return g, H, y


@pytest.mark.parametrize("K", [1, 2, 5])
def test_hand_orthogonal_mmse(golden, K):
    g, H, y = _ortho(golden)
    z, llr = orc.ocd_detect(H, y, g["N0"], g["Es"], K, orc.MMSE, 16)
    zexp = np.array(g["mmse_z_re"]) + 1j * np.array(g["mmse_z_im"])
    assert np.max(np.abs(z[0, 0] - zexp)) < 1e-15
    L0 = [_expr(v) for v in g["mmse_llr_user0"]]
    L1 = [_expr(v) for v in g["mmse_llr_user1"]]
    assert np.max(np.abs(llr[0, 0, 0] - L0)) < 1e-12
    assert np.max(np.abs(llr[0, 0, 1] - L1)) < 1e-12
    mu, rho = orc.exact_mu_rho(H, g["N0"], g["Es"])
    assert np.max(np.abs(mu[0] - g["mmse_mu"])) < 1e-15
    assert np.max(np.abs(rho[0] - g["mmse_rho"])) < 1e-12


def test_hand_orthogonal_box_clips(golden):
    g, H, y = _ortho(golden)
    y = y.copy()
    y[0, 0, 1] = complex(g["box_y2_re"], g["box_y2_im"])
    z, _ = orc.ocd_detect(H, y, g["N0"], g["Es"], 3, orc.BOX, 16)
    zexp = np.array([_expr(v) for v in g["box_z_re"]]) + 1j * np.array(g["box_z_im"])
    assert np.max(np.abs(z[0, 0] - zexp)) < 1e-15


# --------------------------------------------------------------------------
# Invariants and equivalences stated by the paper
# --------------------------------------------------------------------------

def _problem(seed, Nsc=3, B=16, U=4, T=2, order=16, snr=10.0):
    return synth.make_uplink(Nsc, B, U, T, order, snr, seed, dtype=np.complex128)


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_residual_invariant_eq15(mode):
    d = _problem(1, snr=5.0)
    H, Y = d["H"], d["Y"]
    worst = []

    def trace(k, u, z, r):
        ref = Y - np.matmul(z, np.swapaxes(H, 1, 2))
        worst.append(np.max(np.abs(r - ref)) / np.max(np.abs(Y)))

    orc.ocd_equalize(H, Y, d["N0"], 1.0, 4, mode, 16, trace=trace)
    assert len(worst) == 4 * 4 and max(worst) < 1e-12


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
@pytest.mark.parametrize("K", [1, 2, 3, 6])
def test_ocd_equals_plain_cd(mode, K):
    """Section III-B: OCD and CD (Eqs. 12/13) give exactly the same results."""
    d = _problem(2, Nsc=4, B=12, U=5, T=3, snr=3.0)
    z1, *_ = orc.ocd_equalize(d["H"], d["Y"], d["N0"], 1.0, K, mode, 16)
    z2 = orc.cd_equalize(d["H"], d["Y"], d["N0"], 1.0, K, mode, 16)
    assert np.max(np.abs(z1 - z2)) < 1e-12


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_objective_monotone(mode):
    """Each update is an exact coordinate minimisation of Eq. 10."""
    d = _problem(3, Nsc=2, B=8, U=6, T=3, snr=0.0)
    H, Y = d["H"], d["Y"]
    hist = []

    def trace(k, u, z, r):
        hist.append(orc.objective(H, Y, z, d["N0"], 1.0, mode, 16))

    orc.ocd_equalize(H, Y, d["N0"], 1.0, 5, mode, 16, trace=trace)
    f0 = orc.objective(H, Y, np.zeros(Y.shape[:2] + (6,), complex), d["N0"], 1.0, mode, 16)
    prev = f0
    for f in hist:
        assert np.all(np.isfinite(f))
        assert np.all(f <= prev * (1 + 1e-12) + 1e-15)
        prev = f


def test_mmse_converges_to_closed_form():
    """Eqs. 4-5: Gauss-Seidel on the SPD system converges geometrically."""
    d = synth.make_uplink(4, 32, 8, 2, 16, 10.0, 4, dtype=np.complex128)
    ref = orc.mmse_closed_form(d["H"], d["Y"], d["N0"], 1.0)
    errs = []
    for K in (2, 5, 10, 20, 200):
        z, *_ = orc.ocd_equalize(d["H"], d["Y"], d["N0"], 1.0, K, orc.MMSE, 16)
        errs.append(np.max(np.abs(z - ref)) / np.max(np.abs(ref)))
    assert all(a > b for a, b in zip(errs[:-2], errs[1:-1]))
    assert errs[-1] < 1e-10


def test_single_user_one_sweep_is_exact_and_llr_is_exact():
    """U = 1: one sweep solves Eq. 5 and mu~, rho~ equal the exact mu, rho."""
    d = synth.make_uplink(5, 8, 1, 3, 64, 12.0, 5, dtype=np.complex128)
    z, n, dinv, p = orc.ocd_equalize(d["H"], d["Y"], d["N0"], 1.0, 1, orc.MMSE, 64)
    ref = orc.mmse_closed_form(d["H"], d["Y"], d["N0"], 1.0)
    assert np.max(np.abs(z - ref)) < 1e-13
    mu, rho = orc.exact_mu_rho(d["H"], d["N0"], 1.0)
    assert np.max(np.abs(p - mu)) < 1e-14
    assert np.max(np.abs(n / d["N0"] - rho) / rho) < 1e-12
    L_apx = orc.ocd_llr(z, n, p, d["N0"], 1.0, 64)
    L_exact = orc.ocd_llr(z, rho * d["N0"], mu, d["N0"], 1.0, 64)
    assert np.max(np.abs(L_apx - L_exact)) < 1e-9 * max(1.0, np.max(np.abs(L_exact)))


def test_orthogonal_columns_one_sweep_exact():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    Qm, _ = np.linalg.qr(A)
    H = (Qm[:, :4] * np.array([0.5, 1.0, 1.5, 2.0]))[None]
    y = (rng.standard_normal((1, 3, 16)) + 1j * rng.standard_normal((1, 3, 16)))
    z, n, dinv, p = orc.ocd_equalize(H, y, 0.3, 1.0, 1, orc.MMSE, 16)
    ref = orc.mmse_closed_form(H, y, 0.3, 1.0)
    assert np.max(np.abs(z - ref)) < 1e-13
    mu, rho = orc.exact_mu_rho(H, 0.3, 1.0)
    assert np.max(np.abs(p - mu)) < 1e-14


@pytest.mark.parametrize("seed", range(6))
def test_box_matches_bruteforce_qp(seed):
    """Eq. 8 is convex; OCD-BOX at large K reaches its unique minimiser."""
    d = synth.make_uplink(1, 4, 2, 1, 16, -2.0, 100 + seed, dtype=np.complex128)
    H, y = d["H"][0], d["Y"][0, 0]
    zq, fq = orc.box_qp_bruteforce(H, y, 16)
    z, *_ = orc.ocd_equalize(d["H"], d["Y"], d["N0"], 1.0, 2000, orc.BOX, 16)
    assert np.max(np.abs(z[0, 0] - zq)) < 1e-8


def test_box_qp_cases_exercise_the_clip():
    clipped = 0
    a = orc.box_radius(16)
    for seed in range(6):
        d = synth.make_uplink(1, 4, 2, 1, 16, -2.0, 100 + seed, dtype=np.complex128)
        zq, _ = orc.box_qp_bruteforce(d["H"][0], d["Y"][0, 0], 16)
        clipped += np.sum(np.isclose(np.abs(zq.real), a)) + np.sum(np.isclose(np.abs(zq.imag), a))
    assert clipped >= 3


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
@pytest.mark.parametrize("order", [4, 16, 64, 256])
def test_noiseless_recovery(mode, order):
    """B >> U, N0 -> 0: both modes recover s, and the LLR signs give the bits."""
    d = synth.make_noiseless(6, 128, 8, 3, order, seed=7)
    z, llr = orc.ocd_detect(d["H"], d["Y"], 1e-12, 1.0, 60, mode, order)
    assert np.max(np.abs(z - d["S"])) < 1e-6
    assert np.array_equal(orc.hard_bits(llr), d["bits"])


def test_noiseless_recovery_bpsk():
    d = synth.make_noiseless(4, 32, 4, 2, 2, seed=8)
    z, llr = orc.ocd_detect(d["H"], d["Y"], 1e-12, 1.0, 60, orc.BOX, 2)
    assert np.max(np.abs(z.imag)) == 0.0
    assert np.max(np.abs(z - d["S"])) < 1e-6
    assert np.array_equal(orc.hard_bits(llr), d["bits"])


def test_llr_sign_agrees_with_exhaustive_mimo_maxlog():
    """Sanity only: the approximate LLR tracks true MIMO max-log at high SNR."""
    agree = total = 0
    for seed in range(40):
        d = synth.make_uplink(1, 4, 2, 1, 16, 30.0, 200 + seed, dtype=np.complex128)
        _, llr = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 30, orc.MMSE, 16)
        ex = orc.maxlog_mimo_exhaustive(d["H"][0], d["Y"][0, 0], d["N0"], 16)
        agree += np.sum(np.sign(llr[0, 0]) == np.sign(ex))
        total += ex.size
    assert agree / total >= 0.99


@pytest.mark.parametrize("order", [2, 4, 16, 64, 256])
def test_per_dimension_maxlog_equals_exhaustive(order):
    """For a separable Gray alphabet the Eq. 9 minima split per dimension;
    computed here independently, level by level, from the generator's mapping."""
    rng = np.random.default_rng(9)
    z = (rng.standard_normal((2, 3, 4)) + 1j * rng.standard_normal((2, 3, 4))) * 0.8
    n = rng.uniform(0.5, 2.0, (2, 4))
    p = rng.uniform(0.3, 1.0, (2, 4))
    N0 = 0.1
    L = orc.ocd_llr(z, n, p, N0, 1.0, order)
    Q = orc.bits_per_symbol(order)
    x = z / p[:, None, :]
    rho = (n / N0)[:, None, :]
    if order == 2:
        lv = synth.map_bits(np.array([[0], [1]]), 2).real
        ref = rho * ((x.real - lv[0]) ** 2 - (x.real - lv[1]) ** 2)
        assert np.max(np.abs(L[..., 0] - ref)) < 1e-12
        return
    half = Q // 2
    words = np.array(list(itertools.product([0, 1], repeat=half)))
    levels = synth.map_bits(np.concatenate([words, np.zeros_like(words)], axis=1), order).real
    for dim, comp in ((0, x.real), (1, x.imag)):
        dist = (comp[..., None] - levels) ** 2
        for j in range(half):
            d0 = np.min(dist[..., words[:, j] == 0], axis=-1)
            d1 = np.min(dist[..., words[:, j] == 1], axis=-1)
            ref = rho * (d0 - d1)
            assert np.max(np.abs(L[..., dim * half + j] - ref)) < 1e-12


def test_energy_scaling_reading():
    """With E|s|^2 = Es the problem is the unit-energy one on y/sqrt(Es), N0/Es."""
    Es = 2.5
    d = synth.make_uplink(3, 16, 4, 2, 64, 8.0, 10, Es=Es, dtype=np.complex128)
    for mode in (orc.MMSE, orc.BOX):
        z, L = orc.ocd_detect(d["H"], d["Y"], d["N0"], Es, 3, mode, 64)
        z1, L1 = orc.ocd_detect(d["H"], d["Y"] / math.sqrt(Es), d["N0"] / Es, 1.0, 3, mode, 64)
        assert np.max(np.abs(z / math.sqrt(Es) - z1)) < 1e-13
        assert np.max(np.abs(L - L1)) < 1e-10 * max(1.0, np.max(np.abs(L)))


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_zero_column_is_inert(mode):
    """h_u = 0 never touches r: the other users see OCD on H without column u."""
    d = synth.make_uplink(2, 16, 5, 2, 16, 10.0, 11, dtype=np.complex128)
    H = d["H"].copy()
    H[:, :, 2] = 0.0
    z, L = orc.ocd_detect(H, d["Y"], d["N0"], 1.0, 3, mode, 16)
    keep = [0, 1, 3, 4]
    z2, L2 = orc.ocd_detect(H[:, :, keep], d["Y"], d["N0"], 1.0, 3, mode, 16)
    assert np.all(z[:, :, 2] == 0) and np.all(L[:, :, 2] == 0)
    assert np.max(np.abs(z[:, :, keep] - z2)) < 1e-14
    assert np.max(np.abs(L[:, :, keep] - L2)) < 1e-10


def test_zero_sweeps_gives_zero():
    d = _problem(12)
    z, L = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 0, orc.MMSE, 16)
    assert np.all(z == 0)
    assert np.all(np.isfinite(L))


def test_complexity_count_matches_paper():
    """Section III-B: an OCD iteration costs 8BU + 4U real multiplications;
    8BU of them are the inner product and the residual update, i.e. the
    8BUKT real FMAs per subcarrier that the throughput accounting uses."""
    B, U, K, T = 128, 8, 3, 14
    per_iter_mults = 8 * B * U + 4 * U
    inner_and_update = 4 * B * U + 4 * B * U
    assert per_iter_mults - inner_and_update == 4 * U
    assert inner_and_update * K * T == 344064
