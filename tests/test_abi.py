"""The C ABI without a GPU: the library builds, loads, exports every symbol include/dwt2.h
declares, and its host-only queries (layout, workspace size, level limits, argument checks)
behave as documented.  No call here reaches a kernel."""
import ctypes
import os
import re

import pytest

from paper_1708_07853_gb300 import build as B
from paper_1708_07853_gb300 import dwt2 as D
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dwt2_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(D.EXPORTS) | (declared - set(D.EXPORTS))
    assert set(D.EXPORTS) <= declared


def test_status_strings(lib):
    for s in range(7):
        assert lib.dwt2_status_string(s)
    assert lib.dwt2_status_string(99) == b"unknown status"


def test_max_levels_matches_oracle(lib):
    for H, W in [(1, 1), (1, 2), (8, 8), (9, 2), (63, 4096), (8192, 8192), (16384, 3)]:
        assert D.max_levels(H, W) == O.max_levels(H, W)
    assert D.max_levels(0, 5) == 0


@pytest.mark.parametrize("dt", [D.DT_I32, D.DT_F32, D.DT_BF16, D.DT_F16])
def test_layout_shapes_alignment(lib, dt):
    for H, W in [(1, 1), (1, 9), (9, 1), (17, 16), (512, 512), (513, 1000), (8192, 8192)]:
        for lv in sorted({1, D.max_levels(H, W)}):
            bands, nbytes = D.layout(H, W, lv, dt)
            shapes = O.band_shapes(H, W, lv)
            assert len(bands) == len(shapes)
            end = 0
            for b, (kind, j, h, w) in zip(bands, shapes):
                assert (b.h, b.w, b.level) == (h, w, j)
                assert b.kind == {"LL": b"A", "HL": b"H", "LH": b"V", "HH": b"D"}[kind]
                assert b.offset_bytes % 256 == 0 and b.pitch_bytes % 16 == 0
                es = D.ESIZE[b.dtype]
                assert b.pitch_bytes >= w * es
                assert b.offset_bytes >= end  # bands do not overlap
                end = b.offset_bytes + (b.h * b.pitch_bytes if b.h and b.w else 0)
                if kind == "LL":
                    assert b.dtype == (D.DT_I32 if dt == D.DT_I32 else D.DT_F32)
                else:
                    assert b.dtype == dt
            assert nbytes >= end


def test_workspace_bytes(lib):
    n1 = D.workspace_bytes(512, 512, 1, "cdf53", D.DT_F32)
    n3 = D.workspace_bytes(512, 512, 3, "cdf53", D.DT_F32)
    assert n1 == 256
    assert n3 >= 256 + 256 * 256 * 4 + 128 * 128 * 4
    n2p = D.workspace_bytes(512, 512, 3, "cdf53", D.DT_F32, "sep_twopass")
    assert n2p >= n3 + 512 * 512 * 4
    assert lib.dwt2_workspace_bytes(0, 5, 1, 1, 1) == 0
    assert lib.dwt2_workspace_bytes(8, 8, 4, 1, 1) == 0  # too many levels


def test_argument_validation_before_any_launch(lib):
    """Invalid calls are rejected on the host (no pointer is dereferenced, no kernel runs)."""
    fake = ctypes.c_void_p(0x1000)  # never touched: validation fails first
    f = lib.dwt2_forward
    # null image
    assert f(None, 64, 8, 8, 1, fake, fake, 1 << 20, 1, 1, 1, None) == 1
    # too many levels
    assert f(fake, 64, 8, 8, 1, fake, fake, 1 << 20, 1, 4, 1, None) == 1
    # integer wavelet with float storage
    assert f(fake, 64, 8, 8, 1, fake, fake, 1 << 20, 0, 1, 1, None) == 2
    # bf16 image with fp32 bands
    assert f(fake, 64, 8, 8, 2, fake, fake, 1 << 20, 1, 1, 1, None) == 2
    # pitch smaller than a row
    assert f(fake, 16, 8, 8, 1, fake, fake, 1 << 20, 1, 1, 1, None) == 1
    # workspace too small for 3 levels
    assert f(fake, 64, 16, 16, 1, fake, fake, 256, 1, 3, 1, None) == 3
    # unknown scheme
    assert lib.dwt2_forward_scheme(fake, 64, 8, 8, 1, fake, fake, 1 << 20, 1, 1, 1, 7,
                                   None) == 1
    # the adapted scheme (3) has no integer form
    assert lib.dwt2_forward_scheme(fake, 32, 8, 8, 0, fake, fake, 1 << 20, 0, 1, 0, 3,
                                   None) == 2
    # nor the convolution (4)
    assert lib.dwt2_forward_scheme(fake, 32, 8, 8, 0, fake, fake, 1 << 20, 0, 1, 0, 4,
                                   None) == 2
    assert lib.dwt2_forward_scheme(fake, 64, 8, 8, 1, fake, fake, 1 << 20, 1, 1, 1, 5,
                                   None) == 1
    # inverse: null coefficient buffer
    assert lib.dwt2_inverse(None, fake, 64, 8, 8, 1, fake, 1 << 20, 1, 1, 1, None) == 1


def test_batch_validation_and_workspace(lib):
    """Uniform-batch entry points: bad counts and strides are rejected on the host, and the
    workspace holds the shared status header plus one intermediate-LL region per image."""
    fake = ctypes.c_void_p(0x1000)
    one = D.workspace_bytes(512, 512, 3, "cdf97", D.DT_F32)
    for n in (1, 2, 7):
        assert D.workspace_bytes_batch(n, 512, 512, 3, "cdf97", D.DT_F32) == 256 + n * (one - 256)
    assert D.workspace_bytes_batch(5, 512, 512, 1, "cdf97", D.DT_F32) == 256
    assert lib.dwt2_workspace_bytes_batch(0, 8, 8, 1, 1, 1) == 0
    _, cb = D.layout(16, 16, 2, D.DT_F32)
    ws = D.workspace_bytes_batch(4, 16, 16, 2, "cdf97", D.DT_F32)
    f = lib.dwt2_forward_batch
    img_b = 16 * 64
    # N out of range
    assert f(fake, 64, img_b, 0, 16, 16, 1, fake, cb, fake, ws, 2, 2, 1, None) == 1
    assert f(fake, 64, img_b, 70000, 16, 16, 1, fake, cb, fake, ws, 2, 2, 1, None) == 1
    # image batch stride smaller than one image
    assert f(fake, 64, img_b - 64, 4, 16, 16, 1, fake, cb, fake, ws, 2, 2, 1, None) == 1
    # image batch stride not a whole number of elements
    assert f(fake, 64, img_b + 2, 4, 16, 16, 1, fake, cb, fake, ws, 2, 2, 1, None) == 1
    # coefficient batch stride smaller than the layout, or not a multiple of 16
    assert f(fake, 64, img_b, 4, 16, 16, 1, fake, cb - 16, fake, ws, 2, 2, 1, None) == 1
    assert f(fake, 64, img_b, 4, 16, 16, 1, fake, cb + 4, fake, ws, 2, 2, 1, None) == 1
    # workspace sized for fewer images
    small = D.workspace_bytes_batch(3, 16, 16, 2, "cdf97", D.DT_F32)
    assert f(fake, 64, img_b, 4, 16, 16, 1, fake, cb, fake, small, 2, 2, 1, None) == 3
    # the other three directions check the same way
    assert lib.dwt2_inverse_batch(fake, cb + 4, fake, 64, img_b, 4, 16, 16, 1, fake, ws, 2, 2, 1,
                                  None) == 1
    assert lib.dwt2_forward_adjoint_batch(fake, cb, fake, 64, img_b - 64, 4, 16, 16, 1, fake, ws,
                                          2, 2, 1, None) == 1
    assert lib.dwt2_inverse_adjoint_batch(fake, 64, img_b, 0, 16, 16, 1, fake, cb, fake, ws, 2, 2,
                                          1, None) == 1
    # integer wavelet has no adjoint
    assert lib.dwt2_inverse_adjoint_batch(fake, 64, img_b, 4, 16, 16, 0, fake, cb, fake, ws, 0, 2,
                                          0, None) == 2


def test_selftest_validation(lib):
    fake = ctypes.c_void_p(0x1000)
    assert lib.dwt2_selftest_wait_timeout(2, fake, 4096, None) == 1
    assert lib.dwt2_selftest_wait_timeout(0, None, 4096, None) == 1
    assert lib.dwt2_selftest_wait_timeout(0, fake, 128, None) == 1
