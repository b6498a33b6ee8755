"""FP64 reference of the unfolded (differentiable) OCD: Algorithm 1 with a
learnable damping omega_k and regularizer alpha_k per sweep.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the test-suite, the
smoke check and the benchmark's CPU leg may call it; the CUDA library never
does.  Written in plain PyTorch float64 on the CPU so that autograd gives the
reference gradient; nothing here is blocked, fused or reordered.

The paper (arXiv 1611.08779) runs Algorithm 1 with a fixed regularizer and a
plain update.  The unfolded form changes two things per sweep k = 1..K and
keeps everything else of Algorithm 1 and Eq. 9:

    preprocessing of sweep k:  d_{u,k} = 1 / (||h_u||^2 + alpha_k),
                               p_{u,k} = d_{u,k} ||h_u||^2
                               (d = p = 0 when ||h_u||^2 + alpha_k <= 0)
    update of user u:          c   = proj(d_{u,k} h_u^H r + p_{u,k} z_u)
                               dz  = omega_k (c - z_u)
                               z_u <- z_u + dz,   r <- r - h_u dz   (Eq. 15 kept)
    soft output (Eq. 9):       mu~_u = p_{u,K}, rho~_u = ||h_u||^2 Es / N0

With omega_k = 1 and alpha_k = alpha this is Algorithm 1 exactly.  The
projection of Eq. 14 (BOX mode) is written so that its derivative is 1
strictly inside the box and 0 on or outside its bound; the minima of Eq. 9
pass the derivative to the minimizing point.  Loss: binary cross-entropy
with P(b = 1) = sigmoid(L) (L > 0 favours bit 1).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .ocd import BOX, MMSE, alphabet, box_radius


def _project(w: torch.Tensor, mode: int, order: int, Es: float) -> torch.Tensor:
    """Eq. 14 on real and imaginary parts; BPSK zeroes the imaginary part."""
    if mode == MMSE:
        return w
    a = box_radius(order, Es)

    def clip(x):
        return torch.where(x.abs() < a, x, torch.sign(x) * a)

    re = clip(w.real)
    im = torch.zeros_like(w.imag) if order == 2 else clip(w.imag)
    return torch.complex(re, im)


def unfolded_forward(H, Y, N0, Es: float, omega: torch.Tensor, alpha: torch.Tensor,
                     mode: int, order: int, trace=None):
    """Unfolded sweeps for every (subcarrier, symbol).

    H [Nsc, B, U], Y [Nsc, T, B] (complex, any precision; up-cast to
    complex128), N0: scalar or [Nsc], omega and alpha: float64 [K] tensors
    (K >= 1; may require grad).  `trace(k, u, z, r)` is called after every
    user update.  Returns (z [Nsc, T, U], llr [Nsc, T, U, Q]).
    """
    H = torch.as_tensor(np.asarray(H, dtype=np.complex128))
    Y = torch.as_tensor(np.asarray(Y, dtype=np.complex128))
    Nsc, B, U = H.shape
    T = Y.shape[1]
    K = omega.shape[0]
    if K < 1 or alpha.shape[0] != K:
        raise ValueError("omega and alpha need the same length K >= 1")
    N0 = torch.as_tensor(np.broadcast_to(np.asarray(N0, dtype=np.float64), (Nsc,)).copy())
    n = (H.real ** 2 + H.imag ** 2).sum(dim=1)                  # ||h_u||^2, [Nsc, U]
    r = Y.clone()
    z = torch.zeros((Nsc, T, U), dtype=torch.complex128)
    p = None
    for k in range(K):
        den = n + alpha[k]
        d = torch.where(den > 0, 1.0 / torch.where(den > 0, den, torch.ones_like(den)),
                        torch.zeros_like(den))
        p = d * n
        for u in range(U):
            hu = H[:, :, u]                                         # [Nsc, B]
            q = (hu.conj()[:, None, :] * r).sum(dim=2)              # h_u^H r, [Nsc, T]
            w = d[:, u, None] * q + p[:, u, None] * z[:, :, u]
            c = _project(w, mode, order, Es)
            dz = omega[k] * (c - z[:, :, u])
            r = r - hu[:, None, :] * dz[:, :, None]
            z = torch.cat([z[:, :, :u], (z[:, :, u] + dz)[:, :, None], z[:, :, u + 1:]], dim=2)
            if trace is not None:
                trace(k, u, z, r)
    llr = maxlog_llr(z, n, p, N0, Es, order)
    return z, llr


def maxlog_llr(z, n, mu, N0, Es: float, order: int):
    """Eq. 9 with mu~ = mu and rho~ = ||h||^2 Es / N0 (N0 per subcarrier),
    minima over the whole alphabet; users with mu~ = 0 get L = 0."""
    pts_np, lab = alphabet(order, 1.0)
    pts = torch.as_tensor(pts_np)
    mu_b = mu[:, None, :].expand(z.shape)
    rho = (n * Es / N0[:, None])[:, None, :].expand(z.shape)
    ok = mu_b > 0
    x = torch.where(ok, z / torch.where(ok, mu_b, torch.ones_like(mu_b)) / math.sqrt(Es),
                    torch.zeros_like(z))
    dist = (x[..., None] - pts).abs() ** 2                          # [Nsc, T, U, |O|]
    outs = []
    for b in range(lab.shape[1]):
        d0 = dist[..., torch.as_tensor(lab[:, b] == 0)].min(dim=-1).values
        d1 = dist[..., torch.as_tensor(lab[:, b] == 1)].min(dim=-1).values
        outs.append(torch.where(ok, rho * (d0 - d1), torch.zeros_like(rho)))
    return torch.stack(outs, dim=-1)


def bce_loss(llr: torch.Tensor, bits) -> torch.Tensor:
    """Mean binary cross-entropy of the bits under P(b = 1) = sigmoid(L)."""
    b = torch.as_tensor(np.asarray(bits), dtype=llr.dtype)
    return torch.nn.functional.binary_cross_entropy_with_logits(llr, b)


def unfolded_loss_and_grad(H, Y, N0, Es, omega, alpha, mode, order, bits):
    """(loss, d loss / d omega, d loss / d alpha) by reverse-mode autograd in float64."""
    om = torch.as_tensor(np.asarray(omega, dtype=np.float64)).clone().requires_grad_(True)
    al = torch.as_tensor(np.asarray(alpha, dtype=np.float64)).clone().requires_grad_(True)
    _, llr = unfolded_forward(H, Y, N0, Es, om, al, mode, order)
    loss = bce_loss(llr, bits)
    loss.backward()
    return float(loss.detach()), om.grad.numpy().copy(), al.grad.numpy().copy()


__all__ = ["BOX", "MMSE", "unfolded_forward", "maxlog_llr", "bce_loss", "unfolded_loss_and_grad"]
