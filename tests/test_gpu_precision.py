"""Reduced-precision storage: bf16 / fp16 band planes with fp32 lifting arithmetic.

The final LL and the intermediate LL planes stay fp32; only HL / LH / HH are stored in 16 bits
(and, optionally, the input image).  Storing a value v rounds it to nearest, an error of at most
half a unit in the last place: |v| * 2^-9 for bf16 (8 significant bits), |v| * 2^-11 for fp16
(11 significant bits).  The bound used below per element is therefore
    1e-3 (the fp32 bound of the other tests) + |v_oracle| * 2^-p
with p = 8 for bf16 and p = 10 for fp16 (one extra bit of slack for the fp32 value being rounded
not being the oracle's exact value).  fp16 cannot represent magnitudes above 65504; the band
values of [0, 255] inputs stay far below that.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D
from paper_1708_07853_gb300 import inputs as I

from test_gpu_parity import FLOAT_TOL, to_gpu

pytestmark = pytest.mark.gpu

REL = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -10}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _check(got_views, want, dt, what):
    for v, w in zip(got_views, want):
        if w.size == 0:
            continue
        g = v.float().cpu().numpy().astype(np.float64)
        tol = FLOAT_TOL + np.abs(w) * (0.0 if v.dtype == torch.float32 else REL[dt])
        bad = np.abs(g - w) > tol
        assert not bad.any(), (what, np.abs(g - w).max(), np.argwhere(bad)[:3])


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", [(17, 16), (100, 130), (481, 480), (600, 962), (1000, 63)])
def test_16bit_bands_from_fp32_image(dt, wavelet, H, W):
    x = I.field_plus_noise(H, W, I.seed_for(2, H))
    lv = min(5, D.max_levels(H, W))
    c = D.forward(to_gpu(x, torch.float32), wavelet, lv, band_dtype=dt)
    views = c.band_views()
    assert views[0].dtype == torch.float32  # final LL stays fp32
    assert all(v.dtype == dt for v in views[1:])
    _check(views, O.forward(x.astype(np.float64), wavelet, lv), dt, (wavelet, H, W))


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_16bit_image_and_bands(dt, wavelet):
    """A 16-bit image: the oracle transforms the same (already rounded) values."""
    H, W = 517, 300
    x = I.field_plus_noise(H, W, I.seed_for(2, 7))
    t = to_gpu(x, dt)
    xq = t.float().cpu().numpy().astype(np.float64)
    c = D.forward(t, wavelet, 4)
    _check(c.band_views(), O.forward(xq, wavelet, 4), dt, wavelet)


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_16bit_inverse(dt, wavelet):
    """Inverse from 16-bit bands: against the oracle's inverse of the same stored values, to an
    fp32 output and to a 16-bit output (one more rounding of the result)."""
    H, W = 600, 962
    x = I.field_plus_noise(H, W, I.seed_for(2, 8))
    c = D.forward(to_gpu(x, torch.float32), wavelet, 5, band_dtype=dt)
    stored = [v.float().cpu().numpy().astype(np.float64) for v in c.band_views()]
    want = O.inverse(stored, H, W, wavelet, 5)
    r = D.inverse(c, img_dtype=torch.float32).cpu().numpy()
    assert np.abs(r - want).max() <= FLOAT_TOL
    r16 = D.inverse(c, img_dtype=dt).float().cpu().numpy()
    assert (np.abs(r16 - want) <= FLOAT_TOL + np.abs(want) * REL[dt]).all()


def test_16bit_full_size_8192_cdf97():
    x = I.field(8192, 8192, I.seed_for(1))
    t = to_gpu(x, torch.float32)
    want = O.forward(x.astype(np.float64), "cdf97", 5)
    for dt in (torch.bfloat16, torch.float16):
        _check(D.forward(t, "cdf97", 5, band_dtype=dt).band_views(), want, dt, str(dt))
