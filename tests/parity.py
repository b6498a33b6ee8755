"""Tolerances of the GPU-vs-oracle comparison (test infrastructure).

* xhat: max over (w, t) of ||dx||_2 / max(||x_ref||_2, 1e-3 sqrt(U Es)) <= 1e-4.
* LLR:  |dL| <= 1e-3 max(|L_ref|, 1) element-wise.
* hard bits (L > 0): identical, except where the oracle's normalized
  coordinate of that bit's dimension lies within 1e-4 of a PAM decision
  threshold (the midpoints 2k/sigma between levels).
"""
from __future__ import annotations

import math

import numpy as np

import oracle as orc

XHAT_TOL = 1e-4
LLR_REL = 1e-3
BOUNDARY = 1e-4


def xhat_error(x_gpu, x_ref, Es=1.0):
    x_gpu = np.asarray(x_gpu, dtype=np.complex128)
    x_ref = np.asarray(x_ref, dtype=np.complex128)
    U = x_ref.shape[-1]
    num = np.sqrt(np.sum(np.abs(x_gpu - x_ref) ** 2, axis=-1))
    den = np.maximum(np.sqrt(np.sum(np.abs(x_ref) ** 2, axis=-1)), 1e-3 * math.sqrt(U * Es))
    return float(np.max(num / den)) if num.size else 0.0


def llr_excess(L_gpu, L_ref):
    """Largest |dL| / (1e-3 max(|L_ref|, 1)); <= 1 passes."""
    L_gpu = np.asarray(L_gpu, dtype=np.float64)
    L_ref = np.asarray(L_ref, dtype=np.float64)
    if L_ref.size == 0:
        return 0.0
    return float(np.max(np.abs(L_gpu - L_ref) / (LLR_REL * np.maximum(np.abs(L_ref), 1.0))))


def near_threshold_mask(z_ref, p, order, Es=1.0):
    """[..., Q] mask of bits whose dimension sits within BOUNDARY of a threshold."""
    Q = orc.bits_per_symbol(order)
    p = np.broadcast_to(p[:, None, :], z_ref.shape)
    ok = p > 0
    x = np.where(ok, z_ref / np.where(ok, p, 1.0) / math.sqrt(Es), 0.0)
    if order == 2:
        thr = np.array([0.0])
        return (np.min(np.abs(x.real[..., None] - thr), axis=-1) < BOUNDARY)[..., None]
    half = Q // 2
    M = 1 << half
    sigma = math.sqrt(2.0 * (M * M - 1) / 3.0)
    thr = np.array([2.0 * k / sigma for k in range(-(M // 2 - 1), M // 2)])
    near_i = np.min(np.abs(x.real[..., None] - thr), axis=-1) < BOUNDARY
    near_q = np.min(np.abs(x.imag[..., None] - thr), axis=-1) < BOUNDARY
    return np.concatenate([np.repeat(near_i[..., None], half, -1),
                           np.repeat(near_q[..., None], half, -1)], axis=-1)


def hard_bit_mismatches(L_gpu, L_ref, z_ref, p, order, Es=1.0):
    """Number of hard-bit differences outside the threshold neighbourhoods."""
    diff = (np.asarray(L_gpu) > 0) != (np.asarray(L_ref) > 0)
    return int(np.sum(diff & ~near_threshold_mask(np.asarray(z_ref), p, order, Es)))


def assert_parity(x_gpu, L_gpu, H, Y, N0, Es, K, mode, order, label=""):
    z_ref, n, _dinv, p = orc.ocd_equalize(H, Y, N0, Es, K, mode, order)
    report = {}
    if x_gpu is not None:
        report["xhat"] = xhat_error(x_gpu, z_ref, Es)
        assert report["xhat"] <= XHAT_TOL, f"{label} xhat error {report['xhat']:.3e}"
    if L_gpu is not None:
        L_ref = orc.ocd_llr(z_ref, n, p, N0, Es, order)
        report["llr"] = llr_excess(L_gpu, L_ref)
        assert report["llr"] <= 1.0, f"{label} LLR error {report['llr']:.3f} x tolerance"
        report["bits"] = hard_bit_mismatches(L_gpu, L_ref, z_ref, p, order, Es)
        assert report["bits"] == 0, f"{label} {report['bits']} hard-bit mismatches"
    return report
