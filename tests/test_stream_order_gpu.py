"""Stream order with the serialized launches: the detection kernels are
launched with programmatic stream serialization, so their blocks may be
placed while the kernel ahead of them in the stream drains.  Back-to-back
calls into the same outputs, a call whose input a PyTorch kernel writes just
before it, and PyTorch kernels that read the outputs or overwrite the input
just after it, must all see exactly what calls on an idle stream give."""
import pytest

torch = pytest.importorskip("torch")

import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

# (B, U, T, Nsc, algo, 16-bit storage): the bulk-copy kernel with one and two
# user tiles, the one-symbol kernel, the warp-level and the tcgen05 32-user
# kernels, the 16-bit kernel
CASES = [
    (128, 8, 14, 3000, "projected", None),
    (256, 16, 14, 900, "projected", None),
    (128, 8, 1, 20000, "projected", None),
    (128, 32, 14, 600, "projected_warp", None),
    (128, 32, 14, 600, "projected_tc", None),
    (128, 8, 14, 3000, "projected", "bf16"),
]


def stored(x, storage):
    t = torch.from_numpy(x).cuda()
    if storage == "bf16":
        t = torch.view_as_real(t).to(torch.bfloat16).contiguous()
    return t


@pytest.mark.parametrize("B,U,T,Nsc,algo,storage", CASES)
def test_serialized_launches_keep_stream_order(B, U, T, Nsc, algo, storage):
    da = synth.make_uplink(Nsc, B, U, T, 64, 15.0, seed=B + U + T)
    db = synth.make_uplink(Nsc, B, U, T, 64, 12.0, seed=B + U + T + 1)
    H = stored(da["H"], storage)
    Ya = stored(da["Y"], storage)
    Yb = stored(db["Y"], storage)
    N0 = da["N0"]

    def detect(Y, x=None, l=None):
        return ocd.ocd_detect(H, Y, N0, 1.0, 3, "box", 64, xhat=x, llr=l, algo=algo)

    torch.cuda.synchronize()
    x_ref, l_ref = detect(Yb)  # on an idle stream
    torch.cuda.synchronize()
    x_ref, l_ref = x_ref.clone(), l_ref.clone()
    sum_ref = float(torch.view_as_real(x_ref).abs().double().sum())

    # back to back into the same outputs: the second call's results remain
    x = torch.empty_like(x_ref)
    l = torch.empty_like(l_ref)
    detect(Ya, x, l)
    detect(Yb, x, l)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(x), torch.view_as_real(x_ref))
    assert torch.equal(l, l_ref)

    # the input written by a PyTorch kernel just before the call, the outputs
    # read and the input overwritten by PyTorch kernels just after it
    Yc = torch.empty_like(Yb)
    x2 = torch.empty_like(x_ref)
    l2 = torch.empty_like(l_ref)
    torch.cuda.synchronize()
    Yc.copy_(Yb)
    detect(Yc, x2, l2)
    s = torch.view_as_real(x2).abs().double().sum()
    Yc.zero_()
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(x2), torch.view_as_real(x_ref))
    assert torch.equal(l2, l_ref)
    assert float(s) == sum_ref
