"""Failure detection on the GPU without a GPU fault: the bounded wait of the
bulk-copy kernels expires on a barrier nothing completes, the kernel records
the fault and returns, and the context stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as orc  # noqa: E402
import paper_1611_08779_gb300 as ocd  # noqa: E402
from paper_1611_08779_gb300 import _native, synth  # noqa: E402

from .parity import assert_parity  # noqa: E402

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_sets_fault_and_context_survives():
    lib = _native.load()
    ocd.fault_status(clear=True)
    assert lib.ocd_wait_selftest(20000, None) == _native.OCD_OK  # 20 ms limit
    torch.cuda.synchronize()
    assert ocd.fault_status(clear=True) & 1
    assert ocd.fault_status(clear=False) == 0
    # the context still runs the detector correctly afterwards
    d = synth.make_uplink(16, 64, 8, 14, 16, 12.0, 300)
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    x, L = ocd.ocd_detect(H, Y, d["N0"], 1.0, 3, "box", 16, algo="projected")
    torch.cuda.synchronize()
    assert_parity(x.cpu().numpy(), L.cpu().numpy(), d["H"], d["Y"], d["N0"], 1.0, 3,
                  orc.BOX, 16)
    assert ocd.fault_status(clear=False) == 0


def test_selftest_rejects_bad_limits():
    lib = _native.load()
    assert lib.ocd_wait_selftest(0, None) == _native.OCD_ERR_ARG
    assert lib.ocd_wait_selftest(3_000_000, None) == _native.OCD_ERR_ARG


def test_normal_runs_leave_no_fault():
    ocd.fault_status(clear=True)
    d = synth.make_uplink(500, 128, 8, 14, 64, 15.0, 301)
    H = torch.from_numpy(d["H"]).cuda()
    Y = torch.from_numpy(d["Y"]).cuda()
    for _ in range(3):
        ocd.ocd_detect(H, Y, d["N0"], 1.0, 3, "box", 64)
    torch.cuda.synchronize()
    assert ocd.fault_status(clear=False) == 0
    assert np.isfinite(0.0)
