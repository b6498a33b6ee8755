"""FP64 CPU oracle for OCD soft-output MU-MIMO-OFDM detection.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA library: only the test-suite, the smoke check and the benchmark's CPU
baseline leg may import it.  It shares no code with the CUDA path, and the
CUDA path never calls it.

Everything follows Wu, Dick, Cavallaro, Studer, "High-Throughput Data
Detection for Massive MU-MIMO-OFDM using Coordinate Descent" (arXiv
1611.08779).  Each function names the passage it restates.  Arithmetic is
float64 throughout; inputs are up-cast from whatever the caller stores.

Array layouts (row-major): H [Nsc, B, U], Y [Nsc, T, B], z [Nsc, T, U],
LLR [Nsc, T, U, Q].  Loops are vectorised over (subcarrier, symbol) only;
the user order and the sweep order are exactly those of Algorithm 1.

Readings of places where the paper is silent or ambiguous:

* Es: the paper fixes E|s|^2 = 1.  For a general Es the regularizer is
  alpha = N0 / Es, the box radius scales by sqrt(Es), and the LLR is taken on
  z / (mu~ sqrt(Es)) against the unit-energy alphabet with rho~ = ||h||^2 Es / N0.
  With Es = 1 every formula is the paper's.
* Soft output in BOX mode (Section III-C with alpha = 0 gives mu~ = 1 and
  mu~/(1 - mu~) = inf): rho~_u = ||h_u||^2 Es / N0 in both modes.  In MMSE mode
  this equals mu~/(1 - mu~) exactly.
* Gray labelling: first Q/2 bits (MSB first) on the in-phase level, next Q/2
  on the quadrature level, binary-reflected Gray code per dimension.
* LLR sign (Eq. 9 as printed): L = rho (min_{O_b^0} - min_{O_b^1}), so L > 0
  favours bit 1; the hard bit is L > 0 (a tie gives 0).
* Zero column (||h_u||^2 + alpha = 0): d_u^-1 = 0 and p_u = 0, so z_u stays 0,
  and its LLRs are 0.
"""
from __future__ import annotations

import math

import numpy as np

MMSE = 0
BOX = 1


# ---------------------------------------------------------------------------
# Constellation (Section II-A; box radius Section II-D)
# ---------------------------------------------------------------------------

def bits_per_symbol(order: int) -> int:
    if order not in (2, 4, 16, 64, 256):
        raise ValueError(f"unsupported constellation order {order}")
    return int(round(math.log2(order)))


def _gray(i: int) -> int:
    return i ^ (i >> 1)


def alphabet(order: int, Es: float = 1.0):
    """Points of O (E|s|^2 = Es) and their Q-bit labels, MSB first.

    Square QAM: level index i in 0..M-1 has amplitude (2i - (M-1))/sigma with
    sigma^2 = 2(M^2 - 1)/3 (unit average energy, Section II-A) and carries
    the Gray word gray(i).  BPSK: {-1, +1} labelled 0, 1.
    """
    Q = bits_per_symbol(order)
    amp = math.sqrt(Es)
    if order == 2:
        pts = np.array([-amp, amp], dtype=np.complex128)
        lab = np.array([[0], [1]], dtype=np.uint8)
        return pts, lab
    half = Q // 2
    M = 1 << half
    sigma = math.sqrt(2.0 * (M * M - 1) / 3.0)
    pts = []
    labs = []
    for ii in range(M):
        for iq in range(M):
            pts.append(complex((2 * ii - (M - 1)) / sigma, (2 * iq - (M - 1)) / sigma) * amp)
            word = (_gray(ii) << half) | _gray(iq)
            labs.append([(word >> (Q - 1 - b)) & 1 for b in range(Q)])
    return np.array(pts, dtype=np.complex128), np.array(labs, dtype=np.uint8)


def box_radius(order: int, Es: float = 1.0) -> float:
    """alpha = max_{a in O} Re{a}, the radius of the tightest box (Section II-D)."""
    pts, _ = alphabet(order, Es)
    return float(np.max(pts.real))


# ---------------------------------------------------------------------------
# Projection onto C_O (Eq. 14 and the QAM / BPSK special cases after it)
# ---------------------------------------------------------------------------

def project(w: np.ndarray, mode: int, order: int, Es: float = 1.0) -> np.ndarray:
    if mode == MMSE:
        return w
    a = box_radius(order, Es)
    re = np.clip(w.real, -a, a)
    if order == 2:
        return re + 0j
    return re + 1j * np.clip(w.imag, -a, a)


# ---------------------------------------------------------------------------
# Algorithm 1 (OCD)
# ---------------------------------------------------------------------------

def regularizer(mode: int, N0: float, Es: float) -> float:
    """Algorithm 1 initialization: alpha = N0 (MMSE mode) or 0 (BOX mode)."""
    return (N0 / Es) if mode == MMSE else 0.0


def preprocess(H: np.ndarray, N0: float, Es: float, mode: int):
    """Algorithm 1 preprocessing: ||h_u||^2, d_u^-1 = (||h_u||^2 + alpha)^-1, p_u.

    Returns (n, dinv, p), each [Nsc, U] float64.
    """
    H = np.asarray(H, dtype=np.complex128)
    n = np.sum(H.real ** 2 + H.imag ** 2, axis=1)
    denom = n + regularizer(mode, N0, Es)
    with np.errstate(divide="ignore"):
        dinv = np.where(denom > 0.0, 1.0 / np.where(denom > 0.0, denom, 1.0), 0.0)
    p = dinv * n
    return n, dinv, p


def ocd_equalize(H, Y, N0: float, Es: float, K: int, mode: int, order: int,
                 trace=None):
    """Algorithm 1, equalization part, for every (subcarrier, symbol) at once.

    r = y, z = 0; for k = 1..K, for u = 1..U:
        z_u <- proj_C(d_u^-1 h_u^H r + p_u z_u)       (update)
        dz  = z_u(new) - z_u(old)
        r   <- r - h_u dz                               (residual, Eq. 15)
    `trace(k, u, z, r)` (optional) is called after every user update.
    Returns (z [Nsc, T, U], n, dinv, p).
    """
    H = np.asarray(H, dtype=np.complex128)
    Y = np.asarray(Y, dtype=np.complex128)
    Nsc, B, U = H.shape
    T = Y.shape[1]
    n, dinv, p = preprocess(H, N0, Es, mode)
    r = Y.copy()
    z = np.zeros((Nsc, T, U), dtype=np.complex128)
    for k in range(K):
        for u in range(U):
            hu = H[:, :, u]                                   # [Nsc, B]
            c = np.sum(np.conj(hu)[:, None, :] * r, axis=2)   # h_u^H r, [Nsc, T]
            w = dinv[:, u, None] * c + p[:, u, None] * z[:, :, u]
            znew = project(w, mode, order, Es)
            dz = znew - z[:, :, u]
            r = r - hu[:, None, :] * dz[:, :, None]
            z[:, :, u] = znew
            if trace is not None:
                trace(k, u, z, r)
    return z, n, dinv, p


# ---------------------------------------------------------------------------
# Soft output (Eq. 9 with the approximation of Section III-C)
# ---------------------------------------------------------------------------

def ocd_llr(z, n, p, N0: float, Es: float, order: int):
    """Max-log LLRs of Eq. 9 with mu~ = d^-1 g_ii = p and rho~ = ||h||^2 Es / N0.

    The minima run over the whole alphabet (exhaustive, no per-dimension
    shortcut).  Users with mu~ = 0 get L = 0.
    """
    if N0 <= 0.0:
        raise ValueError("soft output needs N0 > 0")
    pts, lab = alphabet(order, 1.0)
    z = np.asarray(z, dtype=np.complex128)
    mu = np.broadcast_to(p[:, None, :], z.shape)
    rho = np.broadcast_to((n * Es / N0)[:, None, :], z.shape)
    ok = mu > 0.0
    x = np.where(ok, z / np.where(ok, mu, 1.0) / math.sqrt(Es), 0.0)
    d = np.abs(x[..., None] - pts) ** 2                     # [Nsc, T, U, |O|]
    Q = lab.shape[1]
    out = np.empty(z.shape + (Q,), dtype=np.float64)
    for b in range(Q):
        d0 = np.min(d[..., lab[:, b] == 0], axis=-1)
        d1 = np.min(d[..., lab[:, b] == 1], axis=-1)
        out[..., b] = rho * (d0 - d1)
    out[~ok] = 0.0
    return out


def ocd_detect(H, Y, N0: float, Es: float, K: int, mode: int, order: int,
               want_llr: bool = True):
    """Whole path: Algorithm 1 then Eq. 9.  Returns (xhat, llr or None)."""
    z, n, _dinv, p = ocd_equalize(H, Y, N0, Es, K, mode, order)
    llr = ocd_llr(z, n, p, N0, Es, order) if want_llr else None
    return z, llr


def hard_bits(llr: np.ndarray) -> np.ndarray:
    """Hard decision from the LLR sign (L > 0 -> bit 1)."""
    return (np.asarray(llr) > 0.0).astype(np.uint8)


# ---------------------------------------------------------------------------
# Independent references used only to pin the functions above
# ---------------------------------------------------------------------------

def objective(H, y, z, N0: float, Es: float, mode: int, order: int) -> np.ndarray:
    """Eq. 10: ||y - Hz||^2 + g(z); g = alpha ||z||^2 (MMSE) or the box indicator."""
    H = np.asarray(H, dtype=np.complex128)
    res = np.asarray(y, dtype=np.complex128) - np.matmul(z, np.swapaxes(H, 1, 2))
    f = np.sum(np.abs(res) ** 2, axis=-1)
    if mode == MMSE:
        f = f + (N0 / Es) * np.sum(np.abs(z) ** 2, axis=-1)
    else:
        a = box_radius(order, Es)
        bad = (np.abs(z.real) > a * (1 + 1e-12)).any(-1) | (np.abs(z.imag) > a * (1 + 1e-12)).any(-1)
        f = np.where(bad, np.inf, f)
    return f


def cd_equalize(H, Y, N0: float, Es: float, K: int, mode: int, order: int):
    """Plain CD, Eqs. 12 (MMSE) and 13 (BOX): every update recomputes
    y - sum_{j != u} h_j z_j from scratch (no residual bookkeeping)."""
    H = np.asarray(H, dtype=np.complex128)
    Y = np.asarray(Y, dtype=np.complex128)
    Nsc, B, U = H.shape
    T = Y.shape[1]
    z = np.zeros((Nsc, T, U), dtype=np.complex128)
    alpha = regularizer(mode, N0, Es)
    for _ in range(K):
        for u in range(U):
            others = [j for j in range(U) if j != u]
            interf = np.matmul(z[:, :, others], np.swapaxes(H[:, :, others], 1, 2))
            e = Y - interf                                     # [Nsc, T, B]
            hu = H[:, :, u]
            nu = np.sum(np.abs(hu) ** 2, axis=1)               # ||h_u||^2
            num = np.sum(np.conj(hu)[:, None, :] * e, axis=2)
            den = (nu + alpha)[:, None]
            w = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
            z[:, :, u] = project(w, mode, order, Es)
    return z


def mmse_closed_form(H, Y, N0: float, Es: float):
    """Eqs. 4-5: z = (G + alpha I)^-1 H^H y with G = H^H H, alpha = N0/Es."""
    H = np.asarray(H, dtype=np.complex128)
    Y = np.asarray(Y, dtype=np.complex128)
    U = H.shape[2]
    Hh = np.conj(np.swapaxes(H, 1, 2))
    A = np.matmul(Hh, H) + (N0 / Es) * np.eye(U)
    mf = np.matmul(Hh, np.swapaxes(Y, 1, 2))                  # [Nsc, U, T]
    return np.swapaxes(np.linalg.solve(A, mf), 1, 2)


def exact_mu_rho(H, N0: float, Es: float):
    """Section II-E: mu_i = [A^-1 G]_ii (row i of A^-1 times column i of G),
    rho_i = mu_i / (1 - mu_i).  Returns (mu, rho), each [Nsc, U]."""
    H = np.asarray(H, dtype=np.complex128)
    U = H.shape[2]
    G = np.matmul(np.conj(np.swapaxes(H, 1, 2)), H)
    A = G + (N0 / Es) * np.eye(U)
    mu = np.real(np.diagonal(np.linalg.solve(A, G), axis1=1, axis2=2))
    return mu, mu / (1.0 - mu)


def box_qp_bruteforce(H, y, order: int, Es: float = 1.0):
    """Exact solution of Eq. 8 for one small problem by active-set enumeration.

    Real form x in R^{2U}; every coordinate is free, at -a or at +a.  For each
    of the 3^{2U} assignments the free part is the least-squares solution with
    the fixed part substituted; the best feasible candidate is the global
    minimizer of this convex problem (the optimum's own active set is one of
    the candidates).  H [B, U], y [B].  QAM only.
    """
    H = np.asarray(H, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    a = box_radius(order, Es)
    B, U = H.shape
    Hr = np.block([[H.real, -H.imag], [H.imag, H.real]])       # [2B, 2U]
    yr = np.concatenate([y.real, y.imag])
    best_f, best_x = np.inf, None
    n = 2 * U
    for code in range(3 ** n):
        state = []
        c = code
        for _ in range(n):
            state.append(c % 3)
            c //= 3
        state = np.array(state)
        free = state == 0
        x = np.where(state == 1, -a, np.where(state == 2, a, 0.0))
        rhs = yr - Hr[:, ~free] @ x[~free]
        if free.any():
            sol, *_ = np.linalg.lstsq(Hr[:, free], rhs, rcond=None)
            if np.any(np.abs(sol) > a * (1 + 1e-12)):
                continue
            x[free] = sol
        f = float(np.sum((yr - Hr @ x) ** 2))
        if f < best_f:
            best_f, best_x = f, x.copy()
    return best_x[:U] + 1j * best_x[U:], best_f


def maxlog_mimo_exhaustive(H, y, N0: float, order: int, Es: float = 1.0):
    """True MIMO max-log LLRs by enumerating O^U (used only as a sanity check):
    L_{u,b} = (min_{s: bit 0} ||y - Hs||^2 - min_{s: bit 1} ||y - Hs||^2) / N0.
    H [B, U], y [B]; returns [U, Q]."""
    H = np.asarray(H, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    pts, lab = alphabet(order, Es)
    B, U = H.shape
    P = len(pts)
    idx = np.indices((P,) * U).reshape(U, -1).T                # [P^U, U]
    S = pts[idx]                                               # [P^U, U]
    m = np.sum(np.abs(y[None, :] - S @ H.T) ** 2, axis=1)      # [P^U]
    Q = lab.shape[1]
    out = np.empty((U, Q))
    for u in range(U):
        for b in range(Q):
            bit = lab[idx[:, u], b]
            out[u, b] = (np.min(m[bit == 0]) - np.min(m[bit == 1])) / N0
    return out
