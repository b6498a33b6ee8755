"""Python binding of the unfolded (differentiable) OCD: torch.autograd.Functions
whose forward and backward are the library's ocd_unfolded_forward /
ocd_unfolded_backward, and ocd_unfolded_bce_forward / ocd_unfolded_bce_backward
for the fused training loss (argument marshalling only).

The learnable parameters are the per-sweep damping omega [K] and regularizer
alpha [K] (float32 CUDA tensors); H, Y and the per-subcarrier noise variance
N0 [Nsc] are data.  Gradients flow to omega and alpha only.
"""
from __future__ import annotations

import torch

from . import _native
from .api import ALGOS, _check_c64, _mode, _stream_handle, bits_per_symbol


def _f32(name, t, n, dev):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or t.device != dev \
            or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be a contiguous float32 tensor of {n} elements on {dev}")


class UnfoldedOCD(torch.autograd.Function):
    """(omega, alpha, H, Y, N0, Es, mode, qam_order, algo) -> (xhat, llr)."""

    @staticmethod
    def forward(ctx, omega, alpha, H, Y, N0, Es=1.0, mode="box", qam_order=16, algo="auto"):
        lib = _native.load()
        _check_c64("H", H)
        _check_c64("Y", Y, H.device)
        dev = H.device
        if dev.type != "cuda":
            raise ValueError("H must be a CUDA tensor (the detector has no CPU path)")
        Nsc, B, U = H.shape
        T = Y.shape[1]
        if tuple(Y.shape) != (Nsc, T, B):
            raise ValueError(f"Y shape {tuple(Y.shape)} does not match H {tuple(H.shape)}")
        K = omega.numel()
        _f32("omega", omega, K, dev)
        _f32("alpha", alpha, K, dev)
        _f32("N0", N0, Nsc, dev)
        Q = bits_per_symbol(qam_order)
        if algo not in ALGOS:
            raise ValueError(f"unknown algo {algo!r}")
        code = ALGOS[algo]
        xhat = torch.empty((Nsc, T, U), dtype=torch.complex64, device=dev)
        llr = torch.empty((Nsc, T, U, Q), dtype=torch.float32, device=dev)
        nck = lib.ocd_unfolded_checkpoint_size(Nsc, B, U, T, K, code)
        ckpt = torch.empty(max(int(nck), 8), dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            st = lib.ocd_unfolded_forward(H.data_ptr(), Y.data_ptr(), Nsc, B, U, T, N0.data_ptr(),
                                          float(Es), K, _mode(mode), int(qam_order),
                                          omega.data_ptr(), alpha.data_ptr(), xhat.data_ptr(),
                                          llr.data_ptr(), ckpt.data_ptr(), code,
                                          _stream_handle(None))
        _native.check(st)
        ctx.save_for_backward(omega, alpha, H, N0, xhat, ckpt)
        ctx.args = (float(Es), _mode(mode), int(qam_order), code)
        # an output the loss does not use gets no zero-filled gradient: its
        # adjoint pointer goes to the library as NULL
        ctx.set_materialize_grads(False)
        return xhat, llr

    @staticmethod
    def backward(ctx, gx, gl):
        lib = _native.load()
        omega, alpha, H, N0, xhat, ckpt = ctx.saved_tensors
        Es, mode, order, code = ctx.args
        Nsc, B, U = H.shape
        T = xhat.shape[1]
        K = omega.numel()
        dev = H.device
        gx = gx.contiguous() if gx is not None else None
        gl = gl.contiguous().float() if gl is not None else None
        domega = torch.empty(K, dtype=torch.float32, device=dev)
        dalpha = torch.empty(K, dtype=torch.float32, device=dev)
        nws = lib.ocd_unfolded_workspace_size(Nsc, T, K)
        ws = torch.empty(max(int(nws), 256), dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            st = lib.ocd_unfolded_backward(H.data_ptr(), Nsc, B, U, T, N0.data_ptr(), Es, K, mode,
                                           order, omega.data_ptr(), alpha.data_ptr(),
                                           xhat.data_ptr(), ckpt.data_ptr(),
                                           gx.data_ptr() if gx is not None else None,
                                           gl.data_ptr() if gl is not None else None,
                                           domega.data_ptr(), dalpha.data_ptr(), ws.data_ptr(),
                                           ws.numel(), code, _stream_handle(None))
        _native.check(st)
        return domega, dalpha, None, None, None, None, None, None, None


def unfolded_ocd(omega, alpha, H, Y, N0, Es=1.0, mode="box", qam_order=16, algo="auto"):
    """Differentiable unfolded OCD: returns (xhat, llr); gradients reach
    omega and alpha through the library's adjoint kernel.  `algo`: "auto",
    "residual" or "projected" (see include/ocd.h)."""
    return UnfoldedOCD.apply(omega, alpha, H, Y, N0, Es, mode, qam_order, algo)


class UnfoldedBCE(torch.autograd.Function):
    """(omega, alpha, H, Y, N0, bits, Es, mode, qam_order, algo) -> (loss,
    xhat, llr): the mean binary cross-entropy of `bits` under P(b = 1) =
    sigmoid(L) over every LLR L, computed where the forward kernel forms the
    LLRs.  Only the loss is differentiable (gradients reach omega and alpha);
    xhat and llr are returned for inspection."""

    @staticmethod
    def forward(ctx, omega, alpha, H, Y, N0, bits, Es=1.0, mode="box", qam_order=16,
                algo="auto"):
        lib = _native.load()
        _check_c64("H", H)
        _check_c64("Y", Y, H.device)
        dev = H.device
        if dev.type != "cuda":
            raise ValueError("H must be a CUDA tensor (the detector has no CPU path)")
        Nsc, B, U = H.shape
        T = Y.shape[1]
        if tuple(Y.shape) != (Nsc, T, B):
            raise ValueError(f"Y shape {tuple(Y.shape)} does not match H {tuple(H.shape)}")
        K = omega.numel()
        _f32("omega", omega, K, dev)
        _f32("alpha", alpha, K, dev)
        _f32("N0", N0, Nsc, dev)
        Q = bits_per_symbol(qam_order)
        _f32("bits", bits, Nsc * T * U * Q, dev)
        if algo not in ALGOS:
            raise ValueError(f"unknown algo {algo!r}")
        code = ALGOS[algo]
        xhat = torch.empty((Nsc, T, U), dtype=torch.complex64, device=dev)
        llr = torch.empty((Nsc, T, U, Q), dtype=torch.float32, device=dev)
        dllr = torch.empty((Nsc, T, U, Q), dtype=torch.float32, device=dev)
        loss = torch.empty((), dtype=torch.float32, device=dev)
        nck = lib.ocd_unfolded_checkpoint_size(Nsc, B, U, T, K, code)
        ckpt = torch.empty(max(int(nck), 8), dtype=torch.uint8, device=dev)
        nws = lib.ocd_unfolded_workspace_size(Nsc, T, K)
        ws = torch.empty(max(int(nws), 256), dtype=torch.uint8, device=dev)
        with torch.cuda.device(dev):
            st = lib.ocd_unfolded_bce_forward(H.data_ptr(), Y.data_ptr(), Nsc, B, U, T,
                                              N0.data_ptr(), float(Es), K, _mode(mode),
                                              int(qam_order), omega.data_ptr(), alpha.data_ptr(),
                                              bits.data_ptr(), xhat.data_ptr(), llr.data_ptr(),
                                              dllr.data_ptr(), loss.data_ptr(), ckpt.data_ptr(),
                                              ws.data_ptr(), ws.numel(), code,
                                              _stream_handle(None))
        _native.check(st)
        ctx.save_for_backward(omega, alpha, H, N0, xhat, ckpt, dllr, ws)
        ctx.args = (float(Es), _mode(mode), int(qam_order), code)
        ctx.mark_non_differentiable(xhat, llr)
        return loss, xhat, llr

    @staticmethod
    def backward(ctx, gloss, gx, gl):
        lib = _native.load()
        omega, alpha, H, N0, xhat, ckpt, dllr, ws = ctx.saved_tensors
        Es, mode, order, code = ctx.args
        Nsc, B, U = H.shape
        T = xhat.shape[1]
        K = omega.numel()
        dev = H.device
        domega = torch.empty(K, dtype=torch.float32, device=dev)
        dalpha = torch.empty(K, dtype=torch.float32, device=dev)
        gs = gloss.to(device=dev, dtype=torch.float32).contiguous() if gloss is not None else None
        with torch.cuda.device(dev):
            st = lib.ocd_unfolded_bce_backward(H.data_ptr(), Nsc, B, U, T, N0.data_ptr(), Es, K,
                                               mode, order, omega.data_ptr(), alpha.data_ptr(),
                                               xhat.data_ptr(), ckpt.data_ptr(), dllr.data_ptr(),
                                               gs.data_ptr() if gs is not None else None,
                                               domega.data_ptr(), dalpha.data_ptr(),
                                               ws.data_ptr(), ws.numel(), code,
                                               _stream_handle(None))
        _native.check(st)
        return domega, dalpha, None, None, None, None, None, None, None, None


def unfolded_bce_loss(omega, alpha, H, Y, N0, bits, Es=1.0, mode="box", qam_order=16,
                      algo="auto", return_outputs=False):
    """Mean binary cross-entropy of `bits` (float32 [Nsc, T, U, Q], labels in
    [0, 1]) under P(b = 1) = sigmoid(L) for the LLRs L of the unfolded OCD,
    fused into the library's forward kernel; loss.backward() runs the
    library's adjoint.  The same value and gradients as
    binary_cross_entropy_with_logits(unfolded_ocd(...)[1], bits) up to float
    rounding.  With return_outputs, returns (loss, xhat, llr)."""
    loss, xhat, llr = UnfoldedBCE.apply(omega, alpha, H, Y, N0, bits, Es, mode, qam_order, algo)
    return (loss, xhat, llr) if return_outputs else loss
