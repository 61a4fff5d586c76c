"""Uniform batches (N images of one size, one launch per level) against the single-image entry
points and the oracle.

Every image of a batch runs the single-image kernel's arithmetic on its own planes (the image
index only selects the planes), so each result must equal the single-image result bit for bit,
for every wavelet, direction and storage type; a sample is also checked against the oracle.
Batch strides that TMA cannot address (not a multiple of 16 bytes) take the plain-load path and
must give the same bits.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D

from test_gpu_parity import FLOAT_TOL, gpu_bands

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _batch(N, H, W, dtype, seed, pad_w=0, pad_img=0):
    """(N, H, W) view into a padded buffer: row pitch W + pad_w, batch stride H*(W+pad_w)+pad_img
    elements."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    per = H * (W + pad_w) + pad_img
    buf = torch.rand(N * per, generator=g, device="cuda") * 255.0
    buf = buf.round().to(torch.int32) if dtype == torch.int32 else buf.to(dtype)
    return buf.as_strided((N, H, W), (per, W + pad_w, 1))


def _coeffs_row(c: torch.Tensor, k, H, W, wavelet, levels, bdt):
    lay, _ = D.layout(H, W, levels, bdt)
    return D.Coeffs(c[k].view(torch.uint8), H, W, D._wid(wavelet), levels, bdt, lay)


def _same(a: D.Coeffs, b: D.Coeffs):
    for x, y in zip(a.band_views(), b.band_views()):
        assert torch.equal(x, y)


CASES = [("cdf53_int", torch.int32, D.DT_I32), ("cdf53", torch.float32, D.DT_F32),
         ("cdf97", torch.float32, D.DT_F32), ("cdf97", torch.float32, D.DT_BF16),
         ("cdf53", torch.float32, D.DT_F16)]
SHAPES = [(5, 256, 256, 4), (3, 517, 300, 3), (7, 33, 1001, 2), (2, 1, 64, 1), (4, 2, 2, 1)]


@pytest.mark.parametrize("wavelet,dtype,bdt", CASES)
@pytest.mark.parametrize("N,H,W,levels", SHAPES)
def test_forward_batch_equals_single_image(wavelet, dtype, bdt, N, H, W, levels):
    x = _batch(N, H, W, dtype, 21)
    c = D.forward_batch(x, wavelet, levels, bdt)
    torch.cuda.synchronize()
    for k in range(N):
        _same(_coeffs_row(c, k, H, W, wavelet, levels, bdt),
              D.forward(x[k], wavelet, levels, band_dtype=bdt))
    if bdt in (D.DT_I32, D.DT_F32):
        k = N - 1
        want = O.forward(x[k].cpu().numpy().astype(np.int64 if dtype == torch.int32 else np.float64),
                         wavelet, levels)
        for gv, w in zip(gpu_bands(_coeffs_row(c, k, H, W, wavelet, levels, bdt)), want):
            if dtype == torch.int32:
                assert np.array_equal(gv, w)
            elif w.size:
                assert np.abs(gv.astype(np.float64) - w).max() <= FLOAT_TOL


@pytest.mark.parametrize("wavelet,dtype,bdt", CASES)
def test_inverse_batch_equals_single_image(wavelet, dtype, bdt):
    N, H, W, levels = 6, 301, 260, 3
    x = _batch(N, H, W, dtype, 22)
    c = D.forward_batch(x, wavelet, levels, bdt)
    y = D.inverse_batch(c, H, W, wavelet, levels, bdt, img_dtype=dtype)
    torch.cuda.synchronize()
    for k in range(N):
        want = D.inverse(_coeffs_row(c, k, H, W, wavelet, levels, bdt), img_dtype=dtype)
        assert torch.equal(y[k], want)
    if dtype == torch.int32:
        assert torch.equal(y, x)


@pytest.mark.parametrize("pad_w,pad_img", [(0, 4), (3, 0), (1, 7)])
def test_unaligned_batch_strides_take_plain_path(pad_w, pad_img):
    """Strides TMA cannot address give the same bits through the plain-load path."""
    N, H, W, levels = 4, 130, 200, 3
    for wavelet, dtype in (("cdf53_int", torch.int32), ("cdf97", torch.float32)):
        x = _batch(N, H, W, dtype, 23, pad_w, pad_img)
        c = D.forward_batch(x, wavelet, levels)
        y = torch.empty(N * (H * (W + pad_w) + pad_img), dtype=dtype, device="cuda").as_strided(
            x.shape, x.stride())
        D.inverse_batch(c, H, W, wavelet, levels, out=y)
        torch.cuda.synchronize()
        for k in range(N):
            _same(_coeffs_row(c, k, H, W, wavelet, levels, D.TORCH_DT[dtype]),
                  D.forward(x[k].contiguous(), wavelet, levels))
            assert torch.equal(y[k], D.inverse(_coeffs_row(c, k, H, W, wavelet, levels,
                                                           D.TORCH_DT[dtype])))


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_adjoint_batches_equal_single_image(wavelet):
    N, H, W, levels = 5, 190, 333, 3
    g = torch.Generator(device="cuda").manual_seed(24)
    gx = torch.randn((N, H, W), generator=g, device="cuda")
    gc = D.inverse_adjoint_batch(gx, wavelet, levels)
    gy = D.forward_adjoint_batch(gc, H, W, wavelet, levels)
    torch.cuda.synchronize()
    for k in range(N):
        ck = _coeffs_row(gc, k, H, W, wavelet, levels, D.DT_F32)
        _same(ck, D.inverse_adjoint(gx[k], wavelet, levels))
        assert torch.equal(gy[k], D.forward_adjoint(ck))


def test_large_batch_and_status():
    """192 images of 1024 x 1024 (the autograd workload's per-call batch), 3 levels of 9/7.
    Launches of this size take the narrow CTA (180-quad strips), single 1024^2 images the wide
    one: every direction must give the single-image bits."""
    N, H, W, levels = 192, 1024, 1024, 3
    x = _batch(N, H, W, torch.float32, 25)
    ws = D.new_workspace(D.workspace_bytes_batch(N, H, W, levels, "cdf97", D.DT_F32), "cuda")
    c = D.forward_batch(x, "cdf97", levels, workspace=ws)
    torch.cuda.synchronize()
    assert D.check_status(ws) == 0
    for k in (0, 77, N - 1):
        _same(_coeffs_row(c, k, H, W, "cdf97", levels, D.DT_F32), D.forward(x[k], "cdf97", levels))
    y = D.inverse_batch(c, H, W, "cdf97", levels)
    torch.cuda.synchronize()
    assert (y - x).abs().max().item() <= FLOAT_TOL
    for k in (0, N - 1):
        assert torch.equal(y[k], D.inverse(_coeffs_row(c, k, H, W, "cdf97", levels, D.DT_F32)))
    # the adjoints of the same batch
    gc = D.inverse_adjoint_batch(y, "cdf97", levels)
    gy = D.forward_adjoint_batch(gc, H, W, "cdf97", levels)
    torch.cuda.synchronize()
    for k in (0, N - 1):
        ck = _coeffs_row(gc, k, H, W, "cdf97", levels, D.DT_F32)
        _same(ck, D.inverse_adjoint(y[k], "cdf97", levels))
        assert torch.equal(gy[k], D.forward_adjoint(ck))


def test_large_int_batch_unaligned_width():
    """64 int32 images of 1000 x 998 (odd band widths, plain loads at level 1 as the pitch is
    not a multiple of 16 bytes), 4 levels of the reversible 5/3: narrow CTAs in the batch, wide
    ones for the single image, the same bits, and an exact round trip."""
    N, H, W, levels = 64, 1000, 998, 4
    x = _batch(N, H, W, torch.int32, 26)
    c = D.forward_batch(x, "cdf53_int", levels)
    y = D.inverse_batch(c, H, W, "cdf53_int", levels)
    torch.cuda.synchronize()
    assert torch.equal(y, x)
    for k in (0, N - 1):
        _same(_coeffs_row(c, k, H, W, "cdf53_int", levels, D.DT_I32),
              D.forward(x[k].contiguous(), "cdf53_int", levels))
    want = O.forward(x[N - 1].cpu().numpy().astype(np.int64), "cdf53_int", levels)
    for gv, w in zip(gpu_bands(_coeffs_row(c, N - 1, H, W, "cdf53_int", levels, D.DT_I32)), want):
        assert np.array_equal(gv, w)
