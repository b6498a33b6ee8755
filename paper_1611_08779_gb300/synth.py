"""Seeded synthetic inputs for the massive MU-MIMO-OFDM uplink (system model, Eq. 1).

This module is the transmit side and the channel only: uniform bits, a Gray
mapping onto a unit-energy square QAM (or BPSK) alphabet, i.i.d. Rayleigh
channels and complex AWGN.  It contains none of the detector's arithmetic
(no equalization, no soft output); both the CUDA path and the FP64 checker
consume what it produces.

Conventions (they fix the labelling a detector must use to recover the bits):

* Alphabet (Section II-A): E|s|^2 = Es, Q = log2 |O| bits per symbol.
* Square QAM with M = 2^(Q/2) levels per real dimension: the first Q/2 bits,
  most significant first, select the in-phase level, the next Q/2 bits the
  quadrature level.  A Q/2-bit group g is a binary-reflected Gray code word;
  its level index is i = gray^-1(g) and the amplitude is
  (2 i - (M - 1)) / sigma * sqrt(Es), sigma^2 = 2 (M^2 - 1) / 3.
* BPSK (|O| = 2, Q = 1): bit 0 -> -sqrt(Es), bit 1 -> +sqrt(Es), imaginary 0.
* Channel: H[w] has i.i.d. CN(0, 1/B) entries, so E ||h_u||^2 = 1.
* Noise: n ~ CN(0, N0) per receive antenna (the paper's n_w lives in C^B; the
  printed C^U is a typo), with N0 = Es * 10^(-SNR_dB / 10), i.e. the SNR is the
  per-user matched-filter SNR.  Eb/N0 in dB is SNR_dB - 10 log10(Q).

Array layouts (row-major, C-contiguous):
    H    complex [Nsc, B, U]
    Y    complex [Nsc, T, B]   (T OFDM symbols share H[w])
    S    complex [Nsc, T, U]   transmitted symbols
    bits uint8   [Nsc, T, U, Q]
"""
from __future__ import annotations

import math

import numpy as np

SUPPORTED_ORDERS = (2, 4, 16, 64, 256)


def bits_per_symbol(order: int) -> int:
    if order not in SUPPORTED_ORDERS:
        raise ValueError(f"unsupported constellation order {order}")
    return int(round(math.log2(order)))


def _gray_to_index(g: np.ndarray) -> np.ndarray:
    """Invert the binary-reflected Gray code word-wise (prefix XOR of the bits)."""
    i = g.copy()
    shift = g >> 1
    while np.any(shift):
        i ^= shift
        shift >>= 1
    return i


def map_bits(bits: np.ndarray, order: int, Es: float = 1.0) -> np.ndarray:
    """Map bit groups (last axis = Q bits, MSB first) to complex symbols."""
    Q = bits_per_symbol(order)
    bits = np.asarray(bits, dtype=np.int64)
    if bits.shape[-1] != Q:
        raise ValueError("last axis must hold Q bits")
    amp = math.sqrt(Es)
    if order == 2:
        return (2.0 * bits[..., 0] - 1.0).astype(np.complex128) * amp
    half = Q // 2
    M = 1 << half
    sigma = math.sqrt(2.0 * (M * M - 1) / 3.0)
    weights = 1 << np.arange(half - 1, -1, -1)
    g_i = (bits[..., :half] * weights).sum(axis=-1)
    g_q = (bits[..., half:] * weights).sum(axis=-1)
    lev_i = _gray_to_index(g_i)
    lev_q = _gray_to_index(g_q)
    re = (2.0 * lev_i - (M - 1)) / sigma
    im = (2.0 * lev_q - (M - 1)) / sigma
    return (re + 1j * im) * amp


def noise_variance(snr_db: float, Es: float = 1.0) -> float:
    return float(Es * 10.0 ** (-snr_db / 10.0))


def make_uplink(Nsc: int, B: int, U: int, T: int, order: int, snr_db: float,
                seed: int, Es: float = 1.0, dtype=np.complex64) -> dict:
    """Draw one batch of uplink data: Y = H S + N (Eq. 1) per subcarrier.

    H and Y are returned in `dtype` (complex64 by default); a consumer that
    wants higher precision should up-cast the stored values so that every
    implementation sees bit-identical inputs.
    """
    if min(Nsc, B, U, T) < 0:
        raise ValueError("sizes must be non-negative")
    Q = bits_per_symbol(order)
    rng = np.random.default_rng(seed)
    scale = math.sqrt(1.0 / (2.0 * B)) if B > 0 else 0.0
    H = (rng.standard_normal((Nsc, B, U)) + 1j * rng.standard_normal((Nsc, B, U))) * scale
    bits = rng.integers(0, 2, size=(Nsc, T, U, Q), dtype=np.uint8)
    S = map_bits(bits, order, Es)
    N0 = noise_variance(snr_db, Es)
    noise = (rng.standard_normal((Nsc, T, B)) + 1j * rng.standard_normal((Nsc, T, B))) \
        * math.sqrt(N0 / 2.0)
    # Y[w, t, :] = H[w] @ S[w, t, :]
    Y = np.matmul(S, np.swapaxes(H, 1, 2)) + noise
    return {
        "H": np.ascontiguousarray(H.astype(dtype)),
        "Y": np.ascontiguousarray(Y.astype(dtype)),
        "S": S,
        "bits": bits,
        "N0": N0,
        "Es": float(Es),
        "order": order,
    }


def make_noiseless(Nsc: int, B: int, U: int, T: int, order: int, seed: int,
                   Es: float = 1.0) -> dict:
    """Same draw as make_uplink but with N = 0 and complex128 storage."""
    d = make_uplink(Nsc, B, U, T, order, snr_db=0.0, seed=seed, Es=Es,
                    dtype=np.complex128)
    d["Y"] = np.ascontiguousarray(np.matmul(d["S"], np.swapaxes(d["H"], 1, 2)))
    d["N0"] = 0.0
    return d


# Cell mix of the batched form: per cell (B, U) from these pairs, a subcarrier
# count uniform in [nsc_lo, nsc_hi], T from MIXED_T, K uniform in [2, 5], MMSE
# or BOX, 16- or 64-QAM, SNR uniform in [snr_lo, snr_hi] dB.
MIXED_BU = ((32, 4), (64, 8), (128, 16), (256, 32))
MIXED_T = (1, 7, 14)


def mixed_cell_specs(ncells: int, seed: int, nsc_lo: int = 300, nsc_hi: int = 3300,
                     snr_lo: float = 5.0, snr_hi: float = 25.0) -> list[dict]:
    """Seeded parameters of `ncells` independent cells; every (B, U) pair and
    every T appear when ncells >= 12 (cells i cycle through the pairs and the
    symbol counts), the rest is drawn."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(ncells):
        B, U = MIXED_BU[i % len(MIXED_BU)]
        T = MIXED_T[(i // len(MIXED_BU)) % len(MIXED_T)]
        specs.append({
            "B": B, "U": U, "T": T,
            "Nsc": int(rng.integers(nsc_lo, nsc_hi + 1)),
            "K": int(rng.integers(2, 6)),
            "mode": "box" if rng.integers(0, 2) else "mmse",
            "order": 64 if rng.integers(0, 2) else 16,
            "snr_db": float(rng.uniform(snr_lo, snr_hi)),
            "seed": int(rng.integers(0, 2**31 - 1)),
        })
    return specs
