"""dwt2_forward_static: the forward transform for callers that cannot allocate device memory.

Such callers (for example code whose host application owns every device allocation and hands
over only the image and the coefficient buffer, or a real-time loop that must never reach the
allocator) cannot provide the workspace that dwt2_forward needs.  dwt2_forward_static uses a
scratch array built into the library instead.  These tests call it through the C ABI and
compare its output with dwt2_forward's on the same input, on two calls in a row (the scratch is
shared between calls and keeps the previous call's contents).

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest
import torch

from paper_1708_07853_gb300 import dwt2 as D
from paper_1708_07853_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DWT2_STATIC_SCRATCH_BYTES = 24 << 20  # include/dwt2.h


@pytest.fixture(scope="module")
def lib():
    from paper_1708_07853_gb300 import build as B
    B.build()
    return D.lib()


def _static_forward(lib, x: torch.Tensor, wavelet: int, levels: int, bdt: int) -> D.Coeffs:
    H, W = x.shape
    c = D.alloc_coeffs(H, W, levels, wavelet, bdt, x.device)
    rc = lib.dwt2_forward_static(x.data_ptr(), x.stride(0) * x.element_size(), H, W,
                                 D.TORCH_DT[x.dtype], c.buffer.data_ptr(), wavelet, levels, bdt,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == 0, (rc, lib.dwt2_last_error())
    return c


@pytest.mark.parametrize("wavelet,dtype,band", [(0, torch.int32, torch.int32),
                                                 (2, torch.float32, torch.float32),
                                                 (2, torch.float32, torch.bfloat16),
                                                 (4, torch.float32, torch.float32)])
def test_static_matches_workspace_entry_point_two_calls(lib, wavelet, dtype, band):
    """Both entry points run the same kernels on the same input, so the coefficients must be the
    same bits; any difference would come from the scratch (an aliased or stale LL plane).  The
    bf16 case keeps its intermediate LL planes in fp32 in the scratch."""
    # two different images, so the second call cannot pass on the first call's leftovers
    for k, (H, W, lv) in enumerate([(1000, 777, 4), (1537, 2049, 5)]):
        x = I.field(H, W, I.seed_for(9, k))
        t = torch.from_numpy(x.astype(np.int32) if dtype == torch.int32 else x).cuda()
        bdt = D.TORCH_DT[band]
        got = _static_forward(lib, t, wavelet, lv, bdt)
        want = D.forward(t, wavelet, lv, band_dtype=band)
        torch.cuda.synchronize()
        for g, w in zip(got.band_views(), want.band_views()):
            assert torch.equal(g, w)


def test_static_rejects_sizes_beyond_its_scratch(lib):
    x = torch.zeros((8192, 8192), dtype=torch.float32, device="cuda")
    c = D.alloc_coeffs(8192, 8192, 1, 2, D.DT_F32, "cuda")
    # one level needs only the status header: accepted at any size
    assert lib.dwt2_forward_static(x.data_ptr(), 8192 * 4, 8192, 8192, D.DT_F32,
                                   c.buffer.data_ptr(), 2, 1, D.DT_F32,
                                   torch.cuda.current_stream().cuda_stream) == 0
    # five levels need two intermediate LL planes (84 MB) > the built-in scratch
    c5 = D.alloc_coeffs(8192, 8192, 5, 2, D.DT_F32, "cuda")
    rc = lib.dwt2_forward_static(x.data_ptr(), 8192 * 4, 8192, 8192, D.DT_F32,
                                 c5.buffer.data_ptr(), 2, 5, D.DT_F32,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == 3  # DWT2_ENOMEM
    assert b"scratch" in lib.dwt2_last_error()
    torch.cuda.synchronize()


def test_static_scratch_limit(lib):
    """4096 x 4096 int32 fits the built-in scratch at the maximum level count; the first square
    size whose workspace exceeds the scratch is rejected with DWT2_ENOMEM before any launch."""
    st = torch.cuda.current_stream().cuda_stream
    n = 4096
    x = torch.from_numpy(I.field(n, n, I.seed_for(9, 5)).astype(np.int32)).cuda()
    lv = D.max_levels(n, n)
    assert lib.dwt2_workspace_bytes(n, n, lv, 0, D.DT_I32) <= DWT2_STATIC_SCRATCH_BYTES
    got = _static_forward(lib, x, 0, lv, D.DT_I32)
    want = D.forward(x, 0, lv)
    torch.cuda.synchronize()
    for g, w in zip(got.band_views(), want.band_views()):
        assert torch.equal(g, w)
    # the first size above the limit (the workspace grows with the size)
    m = n
    while lib.dwt2_workspace_bytes(m, m, 2, 0, D.DT_I32) <= DWT2_STATIC_SCRATCH_BYTES:
        m += 1
    y = torch.zeros((m, m), dtype=torch.int32, device="cuda")
    c = D.alloc_coeffs(m, m, 2, 0, D.DT_I32, "cuda")
    rc = lib.dwt2_forward_static(y.data_ptr(), m * 4, m, m, D.DT_I32, c.buffer.data_ptr(), 0, 2,
                                 D.DT_I32, st)
    assert rc == 3, rc  # DWT2_ENOMEM
    assert b"scratch" in lib.dwt2_last_error()
    torch.cuda.synchronize()
