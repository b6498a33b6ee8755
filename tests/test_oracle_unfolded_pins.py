"""Pins of the FP64 unfolded-OCD reference (oracle/unfolded.py) against what
does not depend on it: the pinned Algorithm 1 oracle (omega = 1, alpha =
Algorithm 1's regularizer), the residual invariant of Eq. 15 under damping,
closed forms for one user, and central finite differences of the loss."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402


def data(Nsc, B, U, T, order, snr, seed):
    return synth.make_uplink(Nsc, B, U, T, order, snr, seed, dtype=np.complex128)


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
@pytest.mark.parametrize("order", [2, 16, 64])
def test_undamped_equals_algorithm_1(mode, order):
    d = data(5, 12, 4, 3, order, 12.0, 11 + order)
    K = 3
    alpha = d["N0"] if mode == orc.MMSE else 0.0
    om = torch.ones(K, dtype=torch.float64)
    al = torch.full((K,), alpha, dtype=torch.float64)
    z, llr = orc.unfolded_forward(d["H"], d["Y"], d["N0"], 1.0, om, al, mode, order)
    z_ref, l_ref = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, K, mode, order)
    assert np.max(np.abs(z.detach().numpy() - z_ref)) < 1e-12
    assert np.max(np.abs(llr.detach().numpy() - l_ref)) < 1e-9 * max(1.0, np.max(np.abs(l_ref)))


def test_residual_invariant_under_damping():
    d = data(3, 10, 3, 2, 16, 8.0, 5)
    H = torch.as_tensor(d["H"])
    Y = torch.as_tensor(d["Y"])
    om = torch.tensor([0.3, 0.9, 1.4], dtype=torch.float64)
    al = torch.tensor([0.5, 0.1, -0.05], dtype=torch.float64)
    worst = [0.0]

    def trace(k, u, z, r):
        res = Y - torch.einsum("wbu,wtu->wtb", H, z)
        worst[0] = max(worst[0], float((r - res).abs().max()))

    orc.unfolded_forward(d["H"], d["Y"], d["N0"], 1.0, om, al, orc.BOX, 16, trace=trace)
    assert worst[0] < 1e-12


def test_one_user_closed_form():
    """U = 1, K = 1, box inactive: z = omega y'h / (||h||^2 + alpha); the
    derivatives follow by hand."""
    rng = np.random.default_rng(3)
    h = (rng.standard_normal((1, 6, 1)) + 1j * rng.standard_normal((1, 6, 1))) * 0.3
    y = (rng.standard_normal((1, 1, 6)) + 1j * rng.standard_normal((1, 1, 6))) * 0.05
    om = torch.tensor([0.7], dtype=torch.float64, requires_grad=True)
    al = torch.tensor([0.2], dtype=torch.float64, requires_grad=True)
    z, _ = orc.unfolded_forward(h, y, 0.1, 1.0, om, al, orc.BOX, 64)
    n = float(np.sum(np.abs(h) ** 2))
    q = complex(np.sum(np.conj(h[0, :, 0]) * y[0, 0]))
    want = 0.7 * q / (n + 0.2)
    assert abs(complex(z[0, 0, 0]) - want) < 1e-14
    assert abs(want.real) < orc.box_radius(64) and abs(want.imag) < orc.box_radius(64)
    z[0, 0, 0].real.backward()
    assert abs(float(om.grad) - (q / (n + 0.2)).real) < 1e-13
    assert abs(float(al.grad) - (-0.7 * q / (n + 0.2) ** 2).real) < 1e-13


def test_clip_derivative_is_zero_outside_the_box():
    """A user driven far outside the box: z is the clip value, its derivative
    with respect to alpha is 0 and with respect to omega is the clip value."""
    h = np.ones((1, 4, 1), dtype=np.complex128)
    y = np.full((1, 1, 4), 10.0 + 0j)
    om = torch.tensor([0.5], dtype=torch.float64, requires_grad=True)
    al = torch.tensor([0.0], dtype=torch.float64, requires_grad=True)
    z, _ = orc.unfolded_forward(h, y, 0.1, 1.0, om, al, orc.BOX, 16)
    a = orc.box_radius(16)
    assert abs(complex(z[0, 0, 0]) - 0.5 * a) < 1e-15
    z[0, 0, 0].real.backward()
    assert abs(float(om.grad) - a) < 1e-15
    assert float(al.grad) == 0.0


@pytest.mark.parametrize("mode", [orc.MMSE, orc.BOX])
def test_gradient_matches_central_differences(mode):
    d = data(4, 16, 4, 3, 16, 10.0, 21)
    N0 = np.array([0.05, 0.1, 0.2, 0.08])
    om = np.array([0.8, 1.1, 0.95])
    al = np.array([0.3, 0.05, 0.12])
    loss, gom, gal = orc.unfolded_loss_and_grad(d["H"], d["Y"], N0, 1.0, om, al, mode, 16,
                                                d["bits"])

    def f(o, a):
        with torch.no_grad():
            _, llr = orc.unfolded_forward(d["H"], d["Y"], N0, 1.0, torch.as_tensor(o),
                                          torch.as_tensor(a), mode, 16)
            return float(orc.bce_loss(llr, d["bits"]))

    eps = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        fd_o = (f(om + e, al) - f(om - e, al)) / (2 * eps)
        fd_a = (f(om, al + e) - f(om, al - e)) / (2 * eps)
        assert abs(fd_o - gom[k]) <= 1e-6 * max(1.0, abs(fd_o)), (k, fd_o, gom[k])
        assert abs(fd_a - gal[k]) <= 1e-6 * max(1.0, abs(fd_a)), (k, fd_a, gal[k])
    assert math.isfinite(loss) and loss > 0


def test_two_sweeps_one_user_closed_form_and_soft_output():
    """U = 1, K = 2, box inactive.  Sweep 1 from z = 0: z1 = omega_1 d_1 q0
    (q0 = h^H y).  Sweep 2: h^H r1 = q0 - n z1, so d_2 h^H r1 + p_2 z1 = d_2 q0
    and z2 = z1 + omega_2 (d_2 q0 - z1).  The soft output uses mu~ = p_2."""
    rng = np.random.default_rng(9)
    h = (rng.standard_normal((1, 8, 1)) + 1j * rng.standard_normal((1, 8, 1))) * 0.35
    y = (rng.standard_normal((1, 1, 8)) + 1j * rng.standard_normal((1, 1, 8))) * 0.05
    om = torch.tensor([0.6, 1.3], dtype=torch.float64)
    al = torch.tensor([0.4, 0.1], dtype=torch.float64)
    z, llr = orc.unfolded_forward(h, y, 0.02, 1.0, om, al, orc.BOX, 16)
    n = float(np.sum(np.abs(h) ** 2))
    q0 = complex(np.sum(np.conj(h[0, :, 0]) * y[0, 0]))
    z1 = 0.6 * q0 / (n + 0.4)
    z2 = z1 + 1.3 * (q0 / (n + 0.1) - z1)
    assert abs(complex(z[0, 0, 0]) - z2) < 1e-14
    p2 = np.array([[n / (n + 0.1)]])
    l_ref = orc.ocd_llr(np.array([[[z2]]]), np.array([[n]]), p2, 0.02, 1.0, 16)
    assert np.max(np.abs(llr.numpy() - l_ref)) < 1e-10


def test_tie_at_the_box_bound_passes_no_gradient():
    """w exactly on the bound (B = U = 1, h = 1, alpha = 0, y = a): the
    projection's derivative there is taken as 0."""
    a = orc.box_radius(16)
    h = np.ones((1, 1, 1), dtype=np.complex128)
    y = np.full((1, 1, 1), a + 0j)
    om = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    al = torch.tensor([0.0], dtype=torch.float64, requires_grad=True)
    z, _ = orc.unfolded_forward(h, y, 0.1, 1.0, om, al, orc.BOX, 16)
    assert complex(z[0, 0, 0]) == a
    z[0, 0, 0].real.backward()
    assert float(al.grad) == 0.0 and float(om.grad) == a


def test_bce_loss_closed_forms():
    """The training loss the fused path reproduces: the mean over all LLRs of
    -log P(b) with P(b = 1) = 1 / (1 + exp(-L)), written out by hand for a
    few logits and labels (L = 0 costs log 2 whatever the label; a confident
    right answer costs almost nothing, a confident wrong one about |L|), and
    its derivative (sigmoid(L) - y) / N."""
    L = torch.tensor([[0.0, 2.0, -3.0], [40.0, -40.0, 0.5]], dtype=torch.float64,
                     requires_grad=True)
    y = np.array([[1, 1, 1], [0, 0, 1]], dtype=np.uint8)
    loss = orc.bce_loss(L, y)
    terms = [math.log(2.0), math.log1p(math.exp(-2.0)), 3.0 + math.log1p(math.exp(-3.0)),
             40.0 + math.log1p(math.exp(-40.0)), math.log1p(math.exp(-40.0)),
             math.log1p(math.exp(-0.5))]
    assert abs(float(loss) - sum(terms) / 6.0) < 1e-14
    loss.backward()
    sig = lambda v: 1.0 / (1.0 + math.exp(-v))  # noqa: E731
    want = [[(sig(0.0) - 1) / 6, (sig(2.0) - 1) / 6, (sig(-3.0) - 1) / 6],
            [sig(40.0) / 6, sig(-40.0) / 6, (sig(0.5) - 1) / 6]]
    assert np.max(np.abs(L.grad.numpy() - np.array(want))) < 1e-15
