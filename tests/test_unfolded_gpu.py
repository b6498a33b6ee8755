"""Unfolded (differentiable) OCD on the GPU: forward values against the FP64
reference of oracle/unfolded.py, gradients of the BCE loss with respect to
the per-sweep damping and regularizer -- each component on its own --
against FP64 autograd, against central differences of the FP64 forward and
of the GPU forward, at small sizes and at the 4096-sample training batch,
and the edge cases of the adjoint."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

from .parity import hard_bit_mismatches, llr_excess, xhat_error  # noqa: E402

pytestmark = pytest.mark.gpu
MODE = {"box": orc.BOX, "mmse": orc.MMSE}


def problem(Nsc, B, U, T, order, seed, snr_lo=5.0, snr_hi=25.0):
    """Per-subcarrier SNR uniform in [snr_lo, snr_hi] dB (N0 per subcarrier)."""
    rng = np.random.default_rng(seed)
    snr = rng.uniform(snr_lo, snr_hi, size=Nsc)
    N0 = 10.0 ** (-snr / 10.0)
    d = synth.make_uplink(Nsc, B, U, T, order, 100.0, seed, dtype=np.complex128)  # noiseless
    noise = (rng.standard_normal(d["Y"].shape) + 1j * rng.standard_normal(d["Y"].shape))
    Y = d["Y"] + noise * np.sqrt(N0 / 2.0)[:, None, None]
    return d["H"].astype(np.complex64), Y.astype(np.complex64), N0.astype(np.float32), d["bits"]


def to_dev(H, Y, N0):
    return torch.from_numpy(H).cuda(), torch.from_numpy(Y).cuda(), torch.from_numpy(N0).cuda()


def params(K, seed):
    rng = np.random.default_rng(seed)
    om = rng.uniform(0.6, 1.3, K).astype(np.float32)
    al = rng.uniform(0.0, 0.3, K).astype(np.float32)
    return om, al


def reference(H, Y, N0, om, al, mode, order, bits=None):
    """FP64 values (and loss gradients when bits are given) on the stored float32 inputs."""
    H64, Y64 = H.astype(np.complex128), Y.astype(np.complex128)
    N064 = N0.astype(np.float64)
    if bits is None:
        with torch.no_grad():
            z, llr = orc.unfolded_forward(H64, Y64, N064, 1.0, torch.as_tensor(om, dtype=torch.float64),
                                          torch.as_tensor(al, dtype=torch.float64), MODE[mode], order)
        return z.numpy(), llr.numpy()
    return orc.unfolded_loss_and_grad(H64, Y64, N064, 1.0, om.astype(np.float64),
                                      al.astype(np.float64), MODE[mode], order, bits)


def gpu_loss_grad(Hd, Yd, N0d, om, al, mode, order, bits_t, arr="auto"):
    o = torch.tensor(om, device="cuda", requires_grad=True)
    a = torch.tensor(al, device="cuda", requires_grad=True)
    x, llr = ocd.unfolded_ocd(o, a, Hd, Yd, N0d, 1.0, mode, order, algo=arr)
    loss = torch.nn.functional.binary_cross_entropy_with_logits(llr, bits_t)
    loss.backward()
    return float(loss), o.grad.cpu().numpy(), a.grad.cpu().numpy()


ARR = ["residual", "projected"]

# Element-wise bound on each gradient component, applied to the omega family
# and to the alpha family separately (the alpha gradients are typically an
# order of magnitude smaller than the omega gradients, so one bound over the
# joined vector would not constrain them):
#     |g_k - g_ref,k| <= GRAD_RTOL * max(|g_ref,k|, GRAD_FLOOR * max_j |g_ref,j|)
# with max_j over the same family.  The GPU forward carries about 1e-6
# relative rounding error per value (FP32, TF32 split products); the adjoint
# replays it and sums per-sample partials in FP32, so a component is good to
# about 1e-5 of the family's scale.  The floor keeps a component that cancels
# to nearly zero from demanding a relative accuracy FP32 cannot give it.
GRAD_RTOL = 2e-3
GRAD_FLOOR = 1e-2


def assert_grad_close(g, g_ref, name):
    g = np.asarray(g, dtype=np.float64)
    g_ref = np.asarray(g_ref, dtype=np.float64)
    floor = GRAD_FLOOR * float(np.max(np.abs(g_ref)))
    bound = GRAD_RTOL * np.maximum(np.abs(g_ref), floor) + 1e-12
    err = np.abs(g - g_ref)
    assert np.all(err <= bound), (
        f"{name}: per-component error / bound = {np.array2string(err / bound, precision=3)}; "
        f"gpu {g}, fp64 {g_ref}")


@pytest.mark.parametrize("arr", ARR)
@pytest.mark.parametrize("mode", ["box", "mmse"])
@pytest.mark.parametrize("B,U,T,K,order", [(128, 16, 2, 5, 16), (32, 8, 3, 3, 64), (33, 5, 4, 2, 4),
                                           (64, 32, 1, 4, 16), (300, 7, 2, 3, 2), (512, 3, 1, 2, 256),
                                           (96, 31, 2, 3, 16), (2, 1, 3, 2, 4)])
def test_forward_matches_the_fp64_reference(mode, B, U, T, K, order, arr):
    H, Y, N0, _ = problem(12, B, U, T, order, seed=B + U + T + K)
    om, al = params(K, seed=K)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    x, llr = ocd.unfolded_ocd(torch.tensor(om, device="cuda"), torch.tensor(al, device="cuda"),
                              Hd, Yd, N0d, 1.0, mode, order, algo=arr)
    torch.cuda.synchronize()
    z_ref, l_ref = reference(H, Y, N0, om, al, mode, order)
    assert xhat_error(x.cpu().numpy(), z_ref) <= 1e-4
    assert llr_excess(llr.cpu().numpy(), l_ref) <= 1.0
    n = np.sum(np.abs(H.astype(np.complex128)) ** 2, axis=1)
    p = n / (n + al[-1])
    assert hard_bit_mismatches(llr.cpu().numpy(), l_ref, z_ref, p, order) == 0


@pytest.mark.parametrize("arr", ARR)
@pytest.mark.parametrize("mode", ["box", "mmse"])
@pytest.mark.parametrize("B,U,T,K,order", [(128, 16, 2, 5, 16), (48, 8, 4, 3, 64), (20, 3, 3, 2, 2),
                                           (64, 32, 1, 3, 16)])
def test_gradients_match_fp64_autograd(mode, B, U, T, K, order, arr):
    H, Y, N0, bits = problem(32, B, U, T, order, seed=7 * B + U)
    om, al = params(K, seed=U + K)
    loss_ref, gom_ref, gal_ref = reference(H, Y, N0, om, al, mode, order, bits)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    loss, gom, gal = gpu_loss_grad(Hd, Yd, N0d, om, al, mode, order, bits_t, arr)
    assert abs(loss - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
    assert_grad_close(gom, gom_ref, "d loss / d omega")
    assert_grad_close(gal, gal_ref, "d loss / d alpha")


@pytest.mark.parametrize("arr", ARR)
def test_gradient_matches_finite_differences_of_the_fp64_forward(arr):
    """Each omega_k and alpha_k gradient of the GPU adjoint against central
    differences of the FP64 forward (step 1e-6: truncation and rounding of
    the difference are both below 1e-8 of the gradient, and a step that small
    crosses no kink of the box or of the max-log minima in practice).  This
    checks the adjoint without going through the reference's autograd."""
    H, Y, N0, bits = problem(96, 64, 8, 2, 16, seed=31)
    om, al = params(4, seed=3)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    _, gom, gal = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, arr)
    H64, Y64, N064 = H.astype(np.complex128), Y.astype(np.complex128), N0.astype(np.float64)

    def f(o, a):
        with torch.no_grad():
            _, llr = orc.unfolded_forward(H64, Y64, N064, 1.0, torch.as_tensor(o),
                                          torch.as_tensor(a), orc.BOX, 16)
            return float(orc.bce_loss(llr, bits))

    eps = 1e-6
    om64, al64 = om.astype(np.float64), al.astype(np.float64)
    fd_o, fd_a = np.zeros(4), np.zeros(4)
    for k in range(4):
        e = np.zeros(4)
        e[k] = eps
        fd_o[k] = (f(om64 + e, al64) - f(om64 - e, al64)) / (2 * eps)
        fd_a[k] = (f(om64, al64 + e) - f(om64, al64 - e)) / (2 * eps)
    assert_grad_close(gom, fd_o, "d loss / d omega vs FP64 differences")
    assert_grad_close(gal, fd_a, "d loss / d alpha vs FP64 differences")


@pytest.mark.parametrize("arr", ARR)
def test_gradient_matches_finite_differences_of_the_gpu_forward(arr):
    """The GPU adjoint against central differences of the GPU forward itself
    (both FP32): a consistency check of the two kernels, not the accuracy
    bound of the adjoint (that is the FP64 comparisons above).  A step small
    enough to cross no kink of the box or of the max-log minima leaves the
    difference of two FP32 losses in rounding noise, and a step above the
    noise crosses kinks; at 2e-3 both are a few percent, so each component is
    held to 3% of itself with a floor of 1e-2.  (At 1024 samples the same
    step gives a 2.6% gap on an alpha gradient of 4e-3 whose GPU value agrees
    with FP64 autograd to 1e-5.)"""
    H, Y, N0, bits = problem(64, 64, 8, 2, 16, seed=31)
    om, al = params(4, seed=3)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    _, gom, gal = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, arr)

    def f(o, a):
        with torch.no_grad():
            _, llr = ocd.unfolded_ocd(torch.tensor(o, device="cuda"), torch.tensor(a, device="cuda"),
                                      Hd, Yd, N0d, 1.0, "box", 16, algo=arr)
            return float(torch.nn.functional.binary_cross_entropy_with_logits(llr.double(), bits_t.double()))

    eps = 2e-3
    for k in range(4):
        e = np.zeros(4, dtype=np.float32)
        e[k] = eps
        fd_o = (f(om + e, al) - f(om - e, al)) / (2 * eps)
        fd_a = (f(om, al + e) - f(om, al - e)) / (2 * eps)
        assert abs(fd_o - gom[k]) <= 3e-2 * max(abs(fd_o), 1e-2), (k, fd_o, gom[k])
        assert abs(fd_a - gal[k]) <= 3e-2 * max(abs(fd_a), 1e-2), (k, fd_a, gal[k])


@pytest.mark.parametrize("arr", ARR)
def test_gradients_at_the_training_batch_size(arr):
    """The unfolded benchmark's configuration: 4096 (subcarrier, symbol)
    samples of 128x16, K = 5, 16-QAM, SNR uniform in 5-25 dB, OCD-BOX, BCE
    loss; same launch partition and gradient reduction as the benchmark
    step.  Every omega_k and alpha_k against FP64 autograd."""
    H, Y, N0, bits = problem(4096, 128, 16, 1, 16, seed=21)
    om, al = params(5, seed=9)
    loss_ref, gom_ref, gal_ref = reference(H, Y, N0, om, al, "box", 16, bits)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    loss, gom, gal = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, arr)
    assert abs(loss - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
    assert_grad_close(gom, gom_ref, "d loss / d omega")
    assert_grad_close(gal, gal_ref, "d loss / d alpha")


def test_gradient_through_xhat_only():
    H, Y, N0, _ = problem(16, 32, 4, 3, 16, seed=41)
    om, al = params(3, seed=4)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    rng = np.random.default_rng(5)
    c = (rng.standard_normal((16, 3, 4)) + 1j * rng.standard_normal((16, 3, 4)))
    o = torch.tensor(om, device="cuda", requires_grad=True)
    a = torch.tensor(al, device="cuda", requires_grad=True)
    x, _ = ocd.unfolded_ocd(o, a, Hd, Yd, N0d, 1.0, "box", 16)
    (x * torch.from_numpy(c.astype(np.complex64)).cuda()).real.sum().backward()
    om64 = torch.tensor(om, dtype=torch.float64, requires_grad=True)
    al64 = torch.tensor(al, dtype=torch.float64, requires_grad=True)
    z, _ = orc.unfolded_forward(H.astype(np.complex128), Y.astype(np.complex128), N0.astype(np.float64),
                                1.0, om64, al64, orc.BOX, 16)
    (z * torch.as_tensor(c)).real.sum().backward()
    assert_grad_close(o.grad.cpu().numpy(), om64.grad.numpy(), "d <c, xhat> / d omega")
    assert_grad_close(a.grad.cpu().numpy(), al64.grad.numpy(), "d <c, xhat> / d alpha")


@pytest.mark.parametrize("arr", ARR)
def test_backward_is_deterministic(arr):
    H, Y, N0, bits = problem(256, 64, 8, 2, 16, seed=51)
    om, al = params(3, seed=6)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    r1 = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, arr)
    r2 = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, arr)
    assert np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])


def test_arrangements_agree():
    """Residual and projected arrangements: same values and gradients up to
    FP32 rounding (identical in exact arithmetic)."""
    H, Y, N0, bits = problem(128, 128, 16, 1, 16, seed=52)
    om, al = params(5, seed=8)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    res = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, "residual")
    prj = gpu_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, "projected")
    assert abs(res[0] - prj[0]) <= 1e-5 * abs(res[0])
    assert_grad_close(prj[1], res[1], "d loss / d omega, projected vs residual")
    assert_grad_close(prj[2], res[2], "d loss / d alpha, projected vs residual")


def test_projected_rejects_a_channel_copy_that_does_not_fit():
    H, Y, N0, _ = problem(2, 512, 32, 1, 16, seed=53)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    with pytest.raises(ocd.OcdError, match="UNSUPPORTED"):
        ocd.unfolded_ocd(torch.ones(2, device="cuda"), torch.zeros(2, device="cuda"), Hd, Yd, N0d,
                         1.0, "box", 16, algo="projected")
    x, _ = ocd.unfolded_ocd(torch.ones(2, device="cuda"), torch.zeros(2, device="cuda"), Hd, Yd, N0d,
                            1.0, "box", 16)  # auto -> residual arrangement
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(torch.view_as_real(x)))


def test_undamped_forward_is_algorithm_1():
    """omega = 1, alpha = 0 in BOX mode is plain OCD-BOX; with one N0 for all
    subcarriers it matches the FP64 Algorithm 1 oracle."""
    d = synth.make_uplink(10, 64, 8, 3, 16, 12.0, 61)
    Hd = torch.from_numpy(d["H"]).cuda()
    Yd = torch.from_numpy(d["Y"]).cuda()
    N0d = torch.full((10,), d["N0"], dtype=torch.float32, device="cuda")
    x, llr = ocd.unfolded_ocd(torch.ones(3, device="cuda"), torch.zeros(3, device="cuda"),
                              Hd, Yd, N0d, 1.0, "box", 16)
    torch.cuda.synchronize()
    z_ref, l_ref = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 3, orc.BOX, 16)
    assert xhat_error(x.cpu().numpy(), z_ref) <= 1e-4
    assert llr_excess(llr.cpu().numpy(), l_ref) <= 1.0


def test_zero_column_and_empty_batch():
    H, Y, N0, bits = problem(6, 16, 4, 2, 16, seed=71)
    H[:, :, 2] = 0
    om, al = params(2, seed=7)
    al[:] = 0.0  # BOX-like: zero column -> d = p = 0
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    o = torch.tensor(om, device="cuda", requires_grad=True)
    a = torch.tensor(al, device="cuda", requires_grad=True)
    x, llr = ocd.unfolded_ocd(o, a, Hd, Yd, N0d, 1.0, "box", 16)
    assert torch.all(x[:, :, 2] == 0) and torch.all(llr[:, :, 2] == 0)
    torch.nn.functional.binary_cross_entropy_with_logits(llr, bits_t).backward()
    assert torch.all(torch.isfinite(o.grad)) and torch.all(torch.isfinite(a.grad))
    # no samples: zero gradients
    He = torch.empty((0, 16, 4), dtype=torch.complex64, device="cuda")
    Ye = torch.empty((0, 2, 16), dtype=torch.complex64, device="cuda")
    o2 = torch.tensor(om, device="cuda", requires_grad=True)
    a2 = torch.tensor(al, device="cuda", requires_grad=True)
    x, llr = ocd.unfolded_ocd(o2, a2, He, Ye, torch.empty(0, device="cuda"), 1.0, "box", 16)
    (llr.sum() + x.real.sum()).backward()
    assert torch.all(o2.grad == 0) and torch.all(a2.grad == 0)


def test_a_few_training_steps_reduce_the_loss():
    """128x16, K = 5, 16-QAM, SNR 5-25 dB: plain gradient steps on omega and
    alpha from a deliberately poor start lower the BCE loss."""
    H, Y, N0, bits = problem(256, 128, 16, 1, 16, seed=81)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    o = torch.full((5,), 0.4, device="cuda", requires_grad=True)
    a = torch.full((5,), 0.5, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([o, a], lr=0.05)
    losses = []
    for _ in range(30):
        opt.zero_grad()
        _, llr = ocd.unfolded_ocd(o, a, Hd, Yd, N0d, 1.0, "box", 16)
        loss = torch.nn.functional.binary_cross_entropy_with_logits(llr, bits_t)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert losses[-1] < 0.8 * losses[0], losses
    assert all(math.isfinite(v) for v in losses)


# ---------------------------------------------------------------------------
# Fused training loss (ocd_unfolded_bce_forward / _backward): the mean BCE of
# the bits and its LLR derivative formed in the forward kernel.
# ---------------------------------------------------------------------------

def fused_loss_grad(Hd, Yd, N0d, om, al, mode, order, bits_t, arr="auto", scale=None):
    o = torch.tensor(om, device="cuda", requires_grad=True)
    a = torch.tensor(al, device="cuda", requires_grad=True)
    loss, x, llr = ocd.unfolded_bce_loss(o, a, Hd, Yd, N0d, bits_t, 1.0, mode, order, algo=arr,
                                         return_outputs=True)
    (loss * scale if scale is not None else loss).backward()
    return float(loss), o.grad.cpu().numpy(), a.grad.cpu().numpy(), x, llr


@pytest.mark.parametrize("arr", ARR)
@pytest.mark.parametrize("mode", ["box", "mmse"])
@pytest.mark.parametrize("B,U,T,K,order", [(128, 16, 2, 5, 16), (48, 8, 4, 3, 64), (20, 3, 3, 2, 2),
                                           (64, 32, 1, 3, 16), (33, 17, 2, 2, 256)])
def test_fused_loss_matches_fp64_autograd(mode, B, U, T, K, order, arr):
    """Loss and every omega_k, alpha_k gradient of the fused path against the
    FP64 reference (oracle/unfolded.py: BCE of the Eq. 9 LLRs), with the
    bound of the composable path.  The shapes reach every forward kernel:
    two samples per warp (U <= 16, projected), one (U > 16, projected) and
    the residual arrangement."""
    H, Y, N0, bits = problem(32, B, U, T, order, seed=11 * B + U)
    om, al = params(K, seed=U + 2 * K)
    loss_ref, gom_ref, gal_ref = reference(H, Y, N0, om, al, mode, order, bits)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    loss, gom, gal, _, _ = fused_loss_grad(Hd, Yd, N0d, om, al, mode, order, bits_t, arr)
    assert abs(loss - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
    assert_grad_close(gom, gom_ref, "d loss / d omega")
    assert_grad_close(gal, gal_ref, "d loss / d alpha")


@pytest.mark.parametrize("arr", ARR)
def test_fused_loss_matches_the_composable_path(arr):
    """Same inputs through unfolded_ocd + binary_cross_entropy_with_logits:
    identical xhat and LLRs (the same kernels form them), the loss and the
    gradients equal up to FP32 rounding (the loss terms are summed in another
    order; d loss / d L = (sigmoid(L) - y) / N is rounded by each side)."""
    H, Y, N0, bits = problem(300, 64, 8, 2, 16, seed=91)
    om, al = params(4, seed=19)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    loss, gom, gal, x, llr = fused_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, arr)
    o = torch.tensor(om, device="cuda", requires_grad=True)
    a = torch.tensor(al, device="cuda", requires_grad=True)
    x2, llr2 = ocd.unfolded_ocd(o, a, Hd, Yd, N0d, 1.0, "box", 16, algo=arr)
    loss2 = torch.nn.functional.binary_cross_entropy_with_logits(llr2, bits_t)
    loss2.backward()
    assert torch.equal(torch.view_as_real(x), torch.view_as_real(x2))
    assert torch.equal(llr, llr2)
    assert abs(loss - float(loss2)) <= 1e-6 * abs(float(loss2))
    np.testing.assert_allclose(gom, o.grad.cpu().numpy(), rtol=1e-4,
                               atol=1e-5 * float(np.max(np.abs(gom))))
    np.testing.assert_allclose(gal, a.grad.cpu().numpy(), rtol=1e-4,
                               atol=1e-5 * float(np.max(np.abs(gal))))


def test_fused_loss_at_the_training_batch_size():
    """The benchmark's training step through the fused path: 4096 samples of
    128x16, K = 5, 16-QAM, SNR 5-25 dB, OCD-BOX; loss and every omega_k,
    alpha_k against FP64 autograd."""
    H, Y, N0, bits = problem(4096, 128, 16, 1, 16, seed=21)
    om, al = params(5, seed=9)
    loss_ref, gom_ref, gal_ref = reference(H, Y, N0, om, al, "box", 16, bits)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    loss, gom, gal, _, _ = fused_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, "projected")
    assert abs(loss - loss_ref) <= 1e-4 * max(1.0, abs(loss_ref))
    assert_grad_close(gom, gom_ref, "d loss / d omega")
    assert_grad_close(gal, gal_ref, "d loss / d alpha")


def test_fused_loss_scales_with_the_incoming_gradient_and_is_deterministic():
    H, Y, N0, bits = problem(256, 64, 8, 2, 16, seed=52)
    om, al = params(3, seed=8)
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    r1 = fused_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t)
    r2 = fused_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t)
    assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1]) and np.array_equal(r1[2], r2[2])
    r3 = fused_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t, scale=-2.5)
    np.testing.assert_allclose(r3[1], -2.5 * r1[1], rtol=1e-6)
    np.testing.assert_allclose(r3[2], -2.5 * r1[2], rtol=1e-6)


def test_fused_loss_edge_cases():
    """A zero channel column gives L = 0 (loss term log 2 per bit) and finite
    gradients; an empty batch gives loss 0 and zero gradients."""
    H, Y, N0, bits = problem(6, 16, 4, 2, 16, seed=72)
    H[:, :, 2] = 0
    om, al = params(2, seed=7)
    al[:] = 0.0
    Hd, Yd, N0d = to_dev(H, Y, N0)
    bits_t = torch.from_numpy(bits.astype(np.float32)).cuda()
    loss, gom, gal, x, llr = fused_loss_grad(Hd, Yd, N0d, om, al, "box", 16, bits_t)
    assert torch.all(llr[:, :, 2] == 0) and math.isfinite(loss)
    assert np.all(np.isfinite(gom)) and np.all(np.isfinite(gal))
    ref = float(torch.nn.functional.binary_cross_entropy_with_logits(llr, bits_t))
    assert abs(loss - ref) <= 1e-6 * ref
    He = torch.empty((0, 16, 4), dtype=torch.complex64, device="cuda")
    Ye = torch.empty((0, 2, 16), dtype=torch.complex64, device="cuda")
    be = torch.empty((0, 2, 4, 4), dtype=torch.float32, device="cuda")
    o = torch.tensor(om, device="cuda", requires_grad=True)
    a = torch.tensor(al, device="cuda", requires_grad=True)
    le = ocd.unfolded_bce_loss(o, a, He, Ye, torch.empty(0, device="cuda"), be, 1.0, "box", 16)
    le.backward()
    assert float(le) == 0.0
    assert torch.all(o.grad == 0) and torch.all(a.grad == 0)
