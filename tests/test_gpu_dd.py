"""GPU parity of the Deslauriers-Dubuc 9/7 and 13/7 wavelets (four-tap lifting steps, the
non-separable scheme of Eq. 5) against the CPU oracle: forward coefficients, the inverse of the
oracle's coefficients and the GPU round trip within 1e-3 on [0, 255] inputs (fp32), ragged and
tiny sizes at every level count, 16-bit band storage within its rounding, unaligned rows, uniform
batches and the 8192^2 five-level workload (plans: test_gpu_batched.py).  The entry points that
do not cover these wavelets (separable comparators, adjoints) must refuse them."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D
from paper_1708_07853_gb300 import inputs as I
from test_gpu_parity import FLOAT_TOL, RAGGED, SMALL, assert_bands, gpu_bands, to_gpu

pytestmark = pytest.mark.gpu

DD = ["dd97", "dd137"]
REL = {torch.bfloat16: 2.0 ** -8, torch.float16: 2.0 ** -10}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _set_oracle_coeffs(H, W, lv, wv, want):
    cc = D.alloc_coeffs(H, W, lv, wv, D.DT_F32, "cuda")
    for v, w in zip(cc.band_views(), want):
        v.copy_(torch.from_numpy(w.astype(np.float32)))
    return cc


def _sizes():
    rng = np.random.default_rng(21)
    extra = [tuple(int(v) for v in rng.integers(1, 700, 2)) for _ in range(4)]
    # planes that take several CTA strips (224 quads) and row blocks, with ragged tails
    return SMALL + RAGGED + extra + [(1030, 1101), (515, 2003)]


@pytest.mark.parametrize("wv", DD)
@pytest.mark.parametrize("H,W", _sizes())
def test_dd_all_levels(wv, H, W):
    rng = np.random.default_rng(H * 13 + W)
    x = rng.uniform(0, 255, (H, W)).astype(np.float32)
    L = D.max_levels(H, W)
    for lv in sorted({1, 2, min(L, 5)} & set(range(1, L + 1))):
        t = to_gpu(x, torch.float32)
        c = D.forward(t, wv, lv)
        want = O.forward(x.astype(np.float64), wv, lv, "eq5")
        assert_bands(gpu_bands(c), want, FLOAT_TOL, ("fwd", wv, H, W, lv))
        r = D.inverse(c).cpu().numpy()
        assert np.abs(r - x).max() <= FLOAT_TOL, ("roundtrip", wv, H, W, lv)
        r2 = D.inverse(_set_oracle_coeffs(H, W, lv, wv, want)).cpu().numpy()
        want_x = O.inverse(want, H, W, wv, lv, "eq5")
        assert np.abs(r2 - want_x).max() <= FLOAT_TOL, ("inv", wv, H, W, lv)


@pytest.mark.parametrize("wv", DD)
def test_dd_constant_image_is_exact(wv):
    """DC gain 1: a constant comes back in LL_J and zeros elsewhere, through the level shift."""
    H, W = 300, 517
    t = torch.full((H, W), 77.0, device="cuda")
    c = D.forward(t, wv, 4)
    views = c.band_views()
    assert torch.all(views[0] == 77.0)
    for v in views[1:]:
        assert torch.all(v == 0)
    assert torch.equal(D.inverse(c), t)


@pytest.mark.parametrize("wv", DD)
@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_dd_16bit_bands(wv, dt):
    H, W = 481, 600
    x = I.field_plus_noise(H, W, I.seed_for(2, H))
    c = D.forward(to_gpu(x, torch.float32), wv, 4, band_dtype=dt)
    want = O.forward(x.astype(np.float64), wv, 4, "eq5")
    for v, w in zip(c.band_views(), want):
        g = v.float().cpu().numpy().astype(np.float64)
        tol = FLOAT_TOL + np.abs(w) * (0.0 if v.dtype == torch.float32 else REL[dt])
        assert np.all(np.abs(g - w) <= tol), (wv, dt, np.abs(g - w).max())


@pytest.mark.parametrize("wv", DD)
@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_dd_16bit_image_and_bands(wv, dt):
    """A 16-bit image: the oracle transforms the same (already rounded) values; the inverse
    writes a 16-bit image within one rounding of the input."""
    H, W = 517, 300
    x = torch.from_numpy(I.field_plus_noise(H, W, I.seed_for(2, W))).to(dt)
    xs = x.float().numpy().astype(np.float64)
    c = D.forward(x.cuda(), wv, 4, band_dtype=dt)
    want = O.forward(xs, wv, 4, "eq5")
    for v, w in zip(c.band_views(), want):
        g = v.float().cpu().numpy().astype(np.float64)
        tol = FLOAT_TOL + np.abs(w) * (0.0 if v.dtype == torch.float32 else REL[dt])
        assert np.all(np.abs(g - w) <= tol), (wv, dt, np.abs(g - w).max())
    # the inverse of the stored (rounded) coefficients, against the oracle's inverse of the same
    # values: fp32 arithmetic plus the rounding of the 16-bit output image
    r = D.inverse(c, img_dtype=dt).float().cpu().numpy().astype(np.float64)
    got = [v.float().cpu().numpy().astype(np.float64) for v in c.band_views()]
    want_r = O.inverse(got, H, W, wv, 4, "eq5")
    assert np.all(np.abs(r - want_r) <= FLOAT_TOL + np.abs(want_r) * REL[dt]), wv


@pytest.mark.parametrize("wv", DD)
def test_dd_unaligned_pitch_matches_aligned(wv):
    H, W = 301, 1517
    x = np.random.default_rng(9).uniform(0, 255, (H, W)).astype(np.float32)
    a = gpu_bands(D.forward(to_gpu(x, torch.float32, pad=0), wv, 3))  # unaligned rows
    b = gpu_bands(D.forward(to_gpu(x, torch.float32, pad=3), wv, 3))  # aligned rows
    assert_bands(a, b, 0, ("pitch", wv))
    c = D.forward(to_gpu(x, torch.float32, pad=3), wv, 3)
    out = torch.zeros((H, W + 1), device="cuda")[:, :W]
    r = D.inverse(c, out=out).cpu().numpy()
    assert np.abs(r - x).max() <= FLOAT_TOL


@pytest.mark.parametrize("wv", DD)
def test_dd_uniform_batch_equals_single_images(wv):
    N, H, W, lv = 6, 257, 390, 3
    xs = torch.rand((N, H, W), device="cuda") * 255
    lay, nbytes = D.layout(H, W, lv, D.DT_F32)
    cb = torch.zeros((N, nbytes // 4), device="cuda")
    ws = D.new_workspace(D.workspace_bytes_batch(N, H, W, lv, wv, D.DT_F32), "cuda")
    D.forward_batch(xs, wv, lv, D.DT_F32, out=cb, workspace=ws)
    y = torch.empty_like(xs)
    D.inverse_batch(cb, H, W, wv, lv, D.DT_F32, out=y, workspace=ws)
    for k in (0, N - 1):
        c = D.forward(xs[k], wv, lv)
        ck = D.Coeffs(cb[k].view(torch.uint8), H, W, D._wid(wv), lv, D.DT_F32, lay)
        for a, b in zip(c.band_views(), ck.band_views()):
            assert torch.equal(a, b), (wv, k)
        assert torch.equal(D.inverse(c), y[k]), (wv, k)


@pytest.mark.parametrize("wv", DD)
def test_dd_full_size_8192_five_levels(wv):
    x = I.field(8192, 8192, I.seed_for(1))
    O.set_threads(16)
    try:
        want = O.forward(x.astype(np.float64), wv, 5, "eq3")  # Eq. 3 = Eq. 5 (oracle pins)
    finally:
        O.set_threads(1)
    t = to_gpu(x, torch.float32)
    c = D.forward(t, wv, 5)
    assert_bands(gpu_bands(c), want, FLOAT_TOL, ("fwd 8192", wv))
    r = D.inverse(c)
    assert (r - t).abs().max().item() <= FLOAT_TOL


@pytest.mark.parametrize("wv", DD)
def test_dd_unsupported_entry_points_refuse(wv):
    x = torch.rand((64, 64), device="cuda")
    with pytest.raises(D.Dwt2Error):
        D.forward(x, wv, 2, scheme="sep_fused")
    with pytest.raises(D.Dwt2Error):
        D.inverse_adjoint(x, wv, 2)
    outs = [D.alloc_coeffs(64, 64, 2, wv, D.DT_F32, "cuda")]
    with pytest.raises(D.Dwt2Error):
        D.Plan([x], outs, wv, 2, "inverse_adjoint", D.DT_F32)
