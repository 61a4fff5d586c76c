"""Out-of-bounds writes, caught with canaries (compute-sanitizer is not available here).

Every byte a call may not write is filled with a sentinel first, then checked afterwards:
- guard regions before and after the coefficient buffer, the image and the workspace;
- the padding inside the coefficient layout (bytes between band rows and between bands);
- the pitch padding of image rows (columns W .. pitch).
The shapes are odd and tiny, and straddle the kernels' tile edges: strips of 240 quad columns
(480 pixels), warp windows of 60 quads, and rows per CTA.  Every direction and scheme is run,
plus uniform batches and plans.  A kernel that stored one element past a row, a band or a plane
would change a sentinel.
"""
import numpy as np
import pytest
import torch

from paper_1708_07853_gb300 import dwt2 as D

pytestmark = pytest.mark.gpu

GUARD = 4096
SENT = 0xA5
SHAPES = [(1, 1), (1, 7), (7, 1), (3, 5), (17, 16), (33, 31), (241, 481), (300, 517),
          (129, 961), (1023, 65)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _guarded(nbytes):
    """(whole, payload): a uint8 buffer with GUARD sentinel bytes on both sides of the payload."""
    whole = torch.full((GUARD + max(nbytes, 16) + GUARD,), SENT, dtype=torch.uint8, device="cuda")
    return whole, whole[GUARD:GUARD + max(nbytes, 16)]


def _guards_intact(whole):
    w = whole.cpu().numpy()
    return (w[:GUARD] == SENT).all() and (w[-GUARD:] == SENT).all()


def _coeffs_guarded(H, W, lv, wavelet, bdt):
    lay, nbytes = D.layout(H, W, lv, bdt)
    whole, payload = _guarded(nbytes)
    return whole, D.Coeffs(payload, H, W, D._wid(wavelet), lv, bdt, lay)


def _padding_intact(c: D.Coeffs):
    """Bytes of the coefficient buffer outside every band's h x w elements still hold SENT."""
    data = c.buffer.cpu().numpy()
    mask = np.zeros(data.size, dtype=bool)
    for b in c.layout:
        es = D.ESIZE[b.dtype]
        for r in range(b.h):
            o = b.offset_bytes + r * b.pitch_bytes
            mask[o:o + b.w * es] = True
    return (data[~mask] == SENT).all()


def _image_guarded(H, W, dtype, aligned=False):
    """An H x W image view with sentinel columns after every row, inside a guarded buffer.
    aligned: the row pitch is a multiple of 16 bytes (vector stores, TMA loads) with at least 4
    padding columns; otherwise 3 padding columns (element stores, plain loads)."""
    es = torch.tensor([], dtype=dtype).element_size()
    pad_cols = 4 + (-(W + 4)) % (16 // es) if aligned else 3
    pitch = (W + pad_cols) * es
    whole, payload = _guarded(H * pitch)
    img = payload[:H * pitch].view(dtype).view(H, W + pad_cols)[:, :W]
    return whole, img


def _pitch_padding_intact(img):
    H, W = img.shape
    full = img.as_strided((H, img.stride(0)), (img.stride(0), 1))
    raw = full[:, W:].contiguous().view(torch.uint8).cpu().numpy()
    return (raw == SENT).all()


def _fill(img, values):
    img.copy_(values)


@pytest.mark.parametrize("wavelet,dtype,bdt", [("cdf53_int", torch.int32, D.DT_I32),
                                               ("cdf53", torch.float32, D.DT_F32),
                                               ("cdf97", torch.float32, D.DT_F32),
                                               ("cdf97", torch.float32, D.DT_BF16)])
@pytest.mark.parametrize("H,W", SHAPES)
def test_forward_inverse_write_nothing_outside(wavelet, dtype, bdt, H, W):
    g = torch.Generator(device="cuda").manual_seed(H * 7 + W)
    lv = min(3, D.max_levels(H, W))
    src = (torch.rand((H, W), generator=g, device="cuda") * 255).to(dtype)
    iw, img = _image_guarded(H, W, dtype)
    _fill(img, src)
    cw, c = _coeffs_guarded(H, W, lv, wavelet, bdt)
    wsb = D.workspace_bytes(H, W, lv, wavelet, bdt)
    ww, ws = _guarded(wsb)
    D.lib().dwt2_workspace_init(ws.data_ptr(), ws.numel(), D._stream_ptr())
    D.forward(img, wavelet, lv, band_dtype=bdt, out=c, workspace=ws[:wsb])
    torch.cuda.synchronize()
    assert _guards_intact(cw) and _padding_intact(c), "forward wrote outside the bands"
    assert _guards_intact(iw) and _pitch_padding_intact(img), "forward wrote to the image"
    assert _guards_intact(ww), "forward wrote past the workspace"
    ow, out = _image_guarded(H, W, dtype, aligned=True)
    D.inverse(c, out=out, workspace=ws[:wsb])
    torch.cuda.synchronize()
    assert _guards_intact(ow) and _pitch_padding_intact(out), "inverse wrote outside the image"
    assert _guards_intact(cw) and _guards_intact(ww)
    if dtype == torch.int32:
        assert torch.equal(out, src)


@pytest.mark.parametrize("scheme", ["sep_fused", "sep_twopass", "adapted", "conv"])
@pytest.mark.parametrize("H,W", SHAPES)
def test_schemes_write_nothing_outside(scheme, H, W):
    g = torch.Generator(device="cuda").manual_seed(H * 5 + W)
    lv = min(3, D.max_levels(H, W))
    iw, img = _image_guarded(H, W, torch.float32)
    _fill(img, torch.rand((H, W), generator=g, device="cuda") * 255)
    cw, c = _coeffs_guarded(H, W, lv, "cdf97", D.DT_F32)
    wsb = D.workspace_bytes(H, W, lv, "cdf97", D.DT_F32, scheme)
    ww, ws = _guarded(wsb)
    D.lib().dwt2_workspace_init(ws.data_ptr(), ws.numel(), D._stream_ptr())
    D.forward(img, "cdf97", lv, scheme=scheme, out=c, workspace=ws[:wsb])
    torch.cuda.synchronize()
    assert _guards_intact(cw) and _padding_intact(c), scheme
    assert _guards_intact(ww) and _guards_intact(iw) and _pitch_padding_intact(img), scheme


@pytest.mark.parametrize("H,W", [(33, 31), (241, 481), (300, 517)])
def test_adjoints_write_nothing_outside(H, W):
    g = torch.Generator(device="cuda").manual_seed(H + W)
    lv = min(3, D.max_levels(H, W))
    iw, gx = _image_guarded(H, W, torch.float32)
    _fill(gx, torch.randn((H, W), generator=g, device="cuda"))
    cw, gc = _coeffs_guarded(H, W, lv, "cdf97", D.DT_F32)
    wsb = D.workspace_bytes(H, W, lv, "cdf97", D.DT_F32)
    ww, ws = _guarded(wsb)
    D.lib().dwt2_workspace_init(ws.data_ptr(), ws.numel(), D._stream_ptr())
    D.inverse_adjoint(gx, "cdf97", lv, out=gc, workspace=ws[:wsb])
    torch.cuda.synchronize()
    assert _guards_intact(cw) and _padding_intact(gc) and _guards_intact(ww)
    ow, out = _image_guarded(H, W, torch.float32, aligned=True)
    D.forward_adjoint(gc, out=out, workspace=ws[:wsb])
    torch.cuda.synchronize()
    assert _guards_intact(ow) and _pitch_padding_intact(out) and _guards_intact(ww)


def test_uniform_batch_writes_nothing_outside():
    N, H, W, lv = 5, 241, 481, 3
    lay, nbytes = D.layout(H, W, lv, D.DT_F32)
    row = (nbytes + 16 + 15) // 16 * 16  # a 16-byte gap of sentinels between images
    whole, payload = _guarded(N * row)
    cbuf = payload[:N * row].view(N, row)
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.rand((N, H, W), generator=g, device="cuda") * 255
    D.forward_batch(x, "cdf97", lv, D.DT_F32, out=cbuf)
    torch.cuda.synchronize()
    assert _guards_intact(whole)
    for k in range(N):
        c = D.Coeffs(cbuf[k], H, W, D._wid("cdf97"), lv, D.DT_F32, lay)
        assert _padding_intact(c), k


def test_plan_writes_nothing_outside():
    sizes = [(241, 481), (33, 31), (1, 7), (300, 517)]
    g = torch.Generator(device="cuda").manual_seed(4)
    imgs, guards = [], []
    for h, w in sizes:
        iw, img = _image_guarded(h, w, torch.float32)
        _fill(img, torch.rand((h, w), generator=g, device="cuda") * 255)
        imgs.append(img)
        guards.append(iw)
    coeffs, cguards = [], []
    for h, w in sizes:
        cw, c = _coeffs_guarded(h, w, 1, "cdf97", D.DT_F32)
        coeffs.append(c)
        cguards.append(cw)
    plan = D.Plan(imgs, coeffs, "cdf97", 1, "forward", D.DT_F32)
    plan.run()
    torch.cuda.synchronize()
    for cw, c in zip(cguards, coeffs):
        assert _guards_intact(cw) and _padding_intact(c)
    outs, oguards = [], []
    for h, w in sizes:
        ow, out = _image_guarded(h, w, torch.float32, aligned=True)
        outs.append(out)
        oguards.append(ow)
    inv = D.Plan(outs, coeffs, "cdf97", 1, "inverse", D.DT_F32)
    inv.run()
    torch.cuda.synchronize()
    for ow, out in zip(oguards, outs):
        assert _guards_intact(ow) and _pitch_padding_intact(out)
