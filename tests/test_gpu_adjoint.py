"""GPU adjoints (transpose lifting) against the fp64 oracle.

The oracle's adjoints are the literal transpose of its transforms (pinned in test_oracle_pins
against dense matrices).  The GPU adjoints compute in fp32, so they are compared with a bound
relative to the size of the result: |gpu - oracle| <= 1e-5 * max(1, max|oracle|) * levels,
fp32 rounding over a few dozen operations per level.  The dot-product identity
<W x, y> = <x, W^T y> is checked on GPU results alone (fp64 accumulation of fp32 values).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (1, 2), (2, 1), (1, 9), (8, 1), (2, 2), (3, 3), (5, 4), (9, 10), (17, 16),
         (16, 17), (33, 31), (100, 130), (481, 480), (600, 962), (37, 1923)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _tol(want, lv):
    m = max((np.abs(w).max() for w in want if np.size(w)), default=1.0)
    return 1e-5 * max(1.0, m) * lv


def _coeffs_from(bands, H, W, wavelet, lv):
    c = D.alloc_coeffs(H, W, lv, wavelet, D.DT_F32, "cuda")
    for v, b in zip(c.band_views(), bands):
        v.copy_(torch.from_numpy(np.asarray(b, dtype=np.float32)))
    return c


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", SIZES)
def test_forward_adjoint_matches_oracle(wavelet, H, W):
    rng = np.random.default_rng(H * 131 + W)
    for lv in sorted({1, min(5, D.max_levels(H, W))}):
        g = [rng.standard_normal((h, w)) for _, _, h, w in O.band_shapes(H, W, lv)]
        got = D.forward_adjoint(_coeffs_from(g, H, W, wavelet, lv)).cpu().numpy()
        want = O.forward_adjoint([x.astype(np.float32).astype(np.float64) for x in g], H, W,
                                 wavelet, lv)
        assert np.abs(got - want).max() <= _tol([want], lv), (H, W, lv)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", SIZES)
def test_inverse_adjoint_matches_oracle(wavelet, H, W):
    rng = np.random.default_rng(H * 17 + W)
    for lv in sorted({1, min(5, D.max_levels(H, W))}):
        g = rng.standard_normal((H, W)).astype(np.float32)
        got = [v.cpu().numpy() for v in D.inverse_adjoint(torch.from_numpy(g).cuda(), wavelet,
                                                          lv).band_views()]
        want = O.inverse_adjoint(g.astype(np.float64), wavelet, lv)
        tol = _tol(want, lv)
        for a, b in zip(got, want):
            if b.size:
                assert np.abs(a - b).max() <= tol, (H, W, lv)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_dot_product_identity_on_gpu(wavelet):
    """<W x, y> = <x, W^T y> and <W^-1 y, x> = <y, W^-T x> from GPU results only."""
    rng = np.random.default_rng(3)
    H, W, lv = 777, 1001, 5
    x = torch.from_numpy(rng.standard_normal((H, W)).astype(np.float32)).cuda()
    y = [rng.standard_normal((h, w)).astype(np.float32) for _, _, h, w in O.band_shapes(H, W, lv)]
    cy = _coeffs_from(y, H, W, wavelet, lv)
    wx = D.forward(x, wavelet, lv)
    lhs = sum(float((a.double() * torch.from_numpy(b).cuda().double()).sum())
              for a, b in zip(wx.band_views(), y))
    rhs = float((x.double() * D.forward_adjoint(cy).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + np.sqrt(H * W))
    winv_y = D.inverse(cy)
    lhs = float((winv_y.double() * x.double()).sum())
    rhs = sum(float((a.double() * torch.from_numpy(b).cuda().double()).sum())
              for a, b in zip(D.inverse_adjoint(x, wavelet, lv).band_views(), y))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + np.sqrt(H * W))


def test_adjoint_rejects_integer_and_16bit():
    x = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(D.Dwt2Error):
        D.inverse_adjoint(x, "cdf53_int", 1)
    c = D.alloc_coeffs(8, 8, 1, "cdf97", D.DT_BF16, "cuda")
    with pytest.raises(D.Dwt2Error):
        D.forward_adjoint(c)
