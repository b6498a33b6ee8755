"""The C-ABI library builds, loads and exports what include/*.h declares, and
rejects invalid arguments on the host before touching a GPU.  No compute
call is made here (these run on machines without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1611_08779_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return _native.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ocd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ocd_detect", "ocd_detect_host", "ocd_last_error", "ocd_version"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    for n in declared_functions():
        assert n in _native.SIGNATURES, f"binding lacks a prototype for {n}"


def test_version(lib):
    assert lib.ocd_version() >= 100


FAKE = 0x10000  # a non-NULL, aligned address that is never dereferenced


def call(lib, H=FAKE, Y=FAKE, Nsc=4, B=16, U=4, T=2, N0=0.1, Es=1.0, K=3, mode=0, order=16,
         xhat=FAKE, llr=FAKE):
    return lib.ocd_detect(H, Y, Nsc, B, U, T, N0, Es, K, mode, order, xhat, llr, None)


@pytest.mark.parametrize("kw,needle", [
    (dict(H=None), "must not be NULL"),
    (dict(Y=None), "must not be NULL"),
    (dict(xhat=None, llr=None), "both outputs"),
    (dict(U=0), "U=0"),
    (dict(U=33), "U=33"),
    (dict(B=0), "B=0"),
    (dict(B=513), "B=513"),
    (dict(K=-1), "K=-1"),
    (dict(K=257), "K=257"),
    (dict(mode=2), "mode"),
    (dict(order=8), "qam_order"),
    (dict(order=32), "qam_order"),
    (dict(Es=0.0), "Es"),
    (dict(Es=float("nan")), "Es"),
    (dict(N0=-1.0), "N0"),
    (dict(N0=float("inf")), "N0"),
    (dict(N0=0.0), "N0 > 0"),
    (dict(Nsc=-1), "Nsc"),
    (dict(T=-1), "T=-1"),
    (dict(H=FAKE + 4), "aligned"),
    (dict(llr=FAKE + 2), "aligned"),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, kw, needle):
    assert call(lib, **kw) == _native.OCD_ERR_ARG
    assert needle in lib.ocd_last_error().decode()


def test_empty_problem_is_a_no_op(lib):
    # Nsc = 0 or T = 0: nothing to enqueue, OK without a device
    assert call(lib, Nsc=0, H=None, Y=None) == _native.OCD_OK
    assert call(lib, T=0, H=None, Y=None) == _native.OCD_OK
    assert call(lib, Nsc=0, H=None, Y=None, xhat=None, llr=None) == _native.OCD_OK


def test_least_squares_without_llr_is_accepted_by_validation(lib):
    # N0 = 0 is legal when only xhat is requested; with no rows it is a no-op
    assert call(lib, N0=0.0, llr=None, Nsc=0) == _native.OCD_OK


def test_host_entry_point_validates(lib):
    st = lib.ocd_detect_host(FAKE, FAKE, 4, 16, 4, 2, 0.1, 1.0, 3, 0, 16, FAKE, FAKE,
                             FAKE, FAKE, FAKE, FAKE, 0, None)
    assert st == _native.OCD_ERR_ARG and "pieces" in lib.ocd_last_error().decode()
    st = lib.ocd_detect_host(FAKE, FAKE, 4, 16, 4, 2, 0.1, 1.0, 3, 0, 16, FAKE, FAKE,
                             None, FAKE, FAKE, FAKE, 2, None)
    assert st == _native.OCD_ERR_ARG and "staging" in lib.ocd_last_error().decode()


def test_fused_loss_entry_points_validate(lib):
    """The fused-loss calls check their extra arguments before any device work."""
    def fwd(bits=FAKE, dllr=FAKE, loss=FAKE, ws=FAKE, ws_bytes=1 << 20):
        return lib.ocd_unfolded_bce_forward(FAKE, FAKE, 4, 16, 4, 2, FAKE, 1.0, 3, 1, 16, FAKE,
                                            FAKE, bits, FAKE, None, dllr, loss, FAKE, ws,
                                            ws_bytes, 0, None)
    assert fwd(loss=None) == _native.OCD_ERR_ARG
    assert "loss must not be NULL" in lib.ocd_last_error().decode()
    for kw in (dict(bits=None), dict(dllr=None)):
        assert fwd(**kw) == _native.OCD_ERR_ARG
        assert "bits and dllr" in lib.ocd_last_error().decode()
    assert fwd(ws_bytes=16) == _native.OCD_ERR_ARG
    assert "workspace" in lib.ocd_last_error().decode()
    assert fwd(bits=FAKE + 2) == _native.OCD_ERR_ARG
    assert "aligned" in lib.ocd_last_error().decode()
    st = lib.ocd_unfolded_bce_backward(FAKE, 4, 16, 4, 2, FAKE, 1.0, 3, 1, 16, FAKE, FAKE, FAKE,
                                       FAKE, None, None, FAKE, FAKE, FAKE, 1 << 20, 0, None)
    assert st == _native.OCD_ERR_ARG and "dllr" in lib.ocd_last_error().decode()


def test_error_message_is_per_thread(lib):
    import threading
    call(lib, U=99)
    seen = {}

    def other():
        call(lib, K=999)
        seen["msg"] = lib.ocd_last_error().decode()

    th = threading.Thread(target=other)
    th.start()
    th.join()
    assert "K=999" in seen["msg"]
    assert "U=99" in lib.ocd_last_error().decode()


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    import paper_1611_08779_gb300 as ocd
    H = torch.zeros((2, 4, 2), dtype=torch.complex64)
    Y = torch.zeros((2, 1, 4), dtype=torch.complex64)
    with pytest.raises(ValueError, match="CUDA"):
        ocd.ocd_detect(H, Y, 0.1)


def test_binding_argument_checks():
    """The binding's own checks (before any library call): alphabets, modes,
    storage types and layouts."""
    torch = pytest.importorskip("torch")
    from paper_1611_08779_gb300 import api
    assert [api.bits_per_symbol(o) for o in (2, 4, 16, 64, 256)] == [1, 2, 4, 6, 8]
    for bad in (8, 32, 1024, 0):
        with pytest.raises(ValueError, match="qam_order"):
            api.bits_per_symbol(bad)
    assert api._mode("BOX") == _native.OCD_BOX and api._mode("mmse") == _native.OCD_MMSE
    with pytest.raises(ValueError, match="mode"):
        api._mode("zf")
    assert api._storage_of("H", torch.zeros((2, 3, 4), dtype=torch.complex64)) == \
        (_native.OCD_STORE_C64, (2, 3, 4))
    assert api._storage_of("H", torch.zeros((2, 3, 4, 2), dtype=torch.bfloat16)) == \
        (_native.OCD_STORE_BF16, (2, 3, 4))
    assert api._storage_of("H", torch.zeros((2, 3, 4, 2), dtype=torch.float16)) == \
        (_native.OCD_STORE_F16, (2, 3, 4))
    with pytest.raises(TypeError, match="expected complex64"):
        api._storage_of("H", torch.zeros((2, 3, 4), dtype=torch.float32))
    with pytest.raises(TypeError, match="expected complex64"):
        api._storage_of("H", torch.zeros((2, 3, 4, 3), dtype=torch.bfloat16))
    with pytest.raises(ValueError, match="contiguous"):
        api._storage_of("H", torch.zeros((4, 3), dtype=torch.complex64).t())
    with pytest.raises(TypeError, match="complex64"):
        api._check_c64("Y", torch.zeros(3, dtype=torch.complex128))


def test_unfolded_bindings_refuse_cpu_tensors():
    """Neither the composable nor the fused-loss unfolded call has a CPU path."""
    torch = pytest.importorskip("torch")
    import paper_1611_08779_gb300 as ocd
    H = torch.zeros((2, 4, 2), dtype=torch.complex64)
    Y = torch.zeros((2, 1, 4), dtype=torch.complex64)
    om = torch.ones(3)
    al = torch.zeros(3)
    N0 = torch.ones(2)
    bits = torch.zeros((2, 1, 2, 4))
    with pytest.raises(ValueError, match="CUDA"):
        ocd.unfolded_ocd(om, al, H, Y, N0, 1.0, "box", 16)
    with pytest.raises(ValueError, match="CUDA"):
        ocd.unfolded_bce_loss(om, al, H, Y, N0, bits, 1.0, "box", 16)


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        saved = _native._lib
        _native._lib = None
        try:
            _native.load(str(tmp_path / "libocd.so"))
        finally:
            _native._lib = saved
