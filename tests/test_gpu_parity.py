"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Bars: the reversible integer CDF 5/3 is bit-exact (forward against the oracle's Eq. 3 order,
inverse = the exact input).  Float results carry fp32 rounding only: on [0, 255] inputs the
maximum absolute error of each GPU result against the fp64 oracle must stay <= 1e-3 at up to
5 levels -- the forward coefficients, the inverse of the oracle's coefficients, and the GPU
round trip inverse(forward(x)) against x.  CDF 5/3 at one level on integer inputs is exact in
fp32 (dyadic coefficients, at most 17 significant bits), so it is compared bit for bit.  The
full-size cases run the benchmark's launch configurations: 8192^2 (int32 5/3 and fp32 9/7) and
16384^2 (fp32 9/7 on the field-plus-noise input), 5 levels, every element against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D
from paper_1708_07853_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FLOAT_TOL = 1e-3  # max abs error of a GPU result vs the oracle, [0, 255] inputs, <= 5 levels


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def to_gpu(x: np.ndarray, dtype, pad: int = 0) -> torch.Tensor:
    """Upload; pad > 0 gives a row pitch of W + pad elements (odd pads make it unaligned)."""
    H, W = x.shape
    t = torch.zeros((H, W + pad), dtype=dtype, device="cuda")
    t[:, :W] = torch.from_numpy(np.ascontiguousarray(x)).to(dtype)
    return t[:, :W]


def gpu_bands(c: D.Coeffs):
    return [v.float().cpu().numpy() if v.dtype != torch.int32 else v.cpu().numpy()
            for v in c.band_views()]


def assert_bands(got, want, tol, what):
    assert len(got) == len(want)
    for k, (g, w) in enumerate(zip(got, want)):
        assert g.shape == w.shape, (what, k, g.shape, w.shape)
        if g.size == 0:
            continue
        if tol == 0:
            bad = np.argwhere(g != w)
            assert bad.size == 0, (what, k, bad[:5], g[tuple(bad[0])], w[tuple(bad[0])])
        else:
            err = np.abs(g.astype(np.float64) - w).max()
            assert err <= tol, (what, k, err)


SMALL = [(1, 1), (1, 2), (2, 1), (1, 7), (7, 1), (2, 2), (3, 3), (5, 4), (4, 5), (9, 10),
         (17, 16), (16, 17), (33, 31)]
RAGGED = [(100, 130), (257, 129), (480, 481), (481, 480), (600, 962), (63, 1000), (1000, 63),
          (37, 1923), (517, 9)]


def _sizes():
    rng = np.random.default_rng(5)
    extra = [tuple(int(v) for v in rng.integers(1, 700, 2)) for _ in range(6)]
    return SMALL + RAGGED + extra


@pytest.mark.parametrize("H,W", _sizes())
def test_int53_bit_exact_all_levels(H, W):
    rng = np.random.default_rng(H * 1000 + W)
    x = rng.integers(-(2 ** 15), 2 ** 15 + 1, (H, W)).astype(np.int32)
    L = D.max_levels(H, W)
    for lv in sorted({1, 2, L} & set(range(1, L + 1))):
        t = to_gpu(x, torch.int32)
        c = D.forward(t, "cdf53_int", lv)
        assert_bands(gpu_bands(c), O.forward(x.astype(np.int64), "cdf53_int", lv), 0,
                     ("fwd", H, W, lv))
        r = D.inverse(c)
        assert torch.equal(r.cpu(), torch.from_numpy(x)), ("inv", H, W, lv)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", _sizes())
def test_float_all_levels(wavelet, H, W):
    rng = np.random.default_rng(H * 7 + W)
    x = rng.uniform(0, 255, (H, W)).astype(np.float32)
    L = D.max_levels(H, W)
    for lv in sorted({1, min(L, 5)}):
        t = to_gpu(x, torch.float32)
        c = D.forward(t, wavelet, lv)
        want = O.forward(x.astype(np.float64), wavelet, lv)
        assert_bands(gpu_bands(c), want, FLOAT_TOL, ("fwd", wavelet, H, W, lv))
        r = D.inverse(c).cpu().numpy()
        assert np.abs(r - x).max() <= FLOAT_TOL, ("roundtrip", wavelet, H, W, lv)
        # inverse of the oracle's own coefficients (inverse checked on its own)
        cc = D.alloc_coeffs(H, W, lv, wavelet, D.DT_F32, "cuda")
        for v, wv in zip(cc.band_views(), want):
            v.copy_(torch.from_numpy(wv.astype(np.float32)))
        r2 = D.inverse(cc).cpu().numpy()
        want_x = O.inverse(want, H, W, wavelet, lv)
        assert np.abs(r2 - want_x).max() <= FLOAT_TOL, ("inv", wavelet, H, W, lv)


# Planes of more than 4 MB (all images of a launch together) take the streaming kernels; smaller
# ones, every case above, the direct kernels.  Ragged shapes just above that size, with aligned
# (TMA) and unaligned (plain-load) rows, for the streaming kernels' edges.
STREAM_RAGGED = [(1201, 1003), (2049, 613), (517, 2311)]


@pytest.mark.parametrize("wavelet", ["cdf53_int", "cdf97"])
@pytest.mark.parametrize("H,W", STREAM_RAGGED)
@pytest.mark.parametrize("pad", [0, 1])
def test_streaming_ragged_above_direct_size(wavelet, H, W, pad):
    rng = np.random.default_rng(H + 3 * W + pad)
    is_int = wavelet == "cdf53_int"
    dt = torch.int32 if is_int else torch.float32
    x = (rng.integers(-(2 ** 15), 2 ** 15 + 1, (H, W)).astype(np.int32) if is_int
         else rng.uniform(0, 255, (H, W)).astype(np.float32))
    for lv in (1, 3):
        c = D.forward(to_gpu(x, dt, pad), wavelet, lv)
        want = O.forward(x.astype(np.int64 if is_int else np.float64), wavelet, lv)
        assert_bands(gpu_bands(c), want, 0 if is_int else FLOAT_TOL, ("fwd", wavelet, H, W, lv))
        out = torch.zeros((H, W + pad), dtype=dt, device="cuda")[:, :W]
        r = D.inverse(c, out=out).cpu().numpy()
        if is_int:
            assert (r == x).all(), ("inv", H, W, lv)
        else:
            assert np.abs(r - x).max() <= FLOAT_TOL, ("roundtrip", H, W, lv)


def test_cdf53_float_one_level_exact_config_512():
    """512 x 512 integer field in [0, 255], float CDF 5/3, one level: exact in fp32."""
    x = I.field(512, 512, I.seed_for(0))
    t = to_gpu(x, torch.float32)
    c = D.forward(t, "cdf53", 1)
    want = O.forward(x.astype(np.float64), "cdf53", 1)
    assert_bands(gpu_bands(c), want, 0, "fwd 512")
    r = D.inverse(c).cpu().numpy()
    assert (r == x).all()


@pytest.mark.parametrize("wavelet", ["cdf53_int", "cdf53", "cdf97"])
def test_unaligned_pitch_matches_aligned(wavelet):
    """Rows whose pitch is not a multiple of 16 bytes take the plain-load path; same results."""
    H, W = 301, 517
    rng = np.random.default_rng(9)
    dt = torch.int32 if wavelet == "cdf53_int" else torch.float32
    x = rng.integers(0, 256, (H, W)).astype(np.int32 if dt == torch.int32 else np.float32)
    a = gpu_bands(D.forward(to_gpu(x, dt, pad=0), wavelet, 3))  # pitch 517*4: unaligned
    b = gpu_bands(D.forward(to_gpu(x, dt, pad=3), wavelet, 3))  # pitch 520*4: aligned
    assert_bands(a, b, 0, "pitch")
    c = D.forward(to_gpu(x, dt, pad=3), wavelet, 3)
    out = torch.zeros((H, W + 1), dtype=dt, device="cuda")[:, :W]  # unaligned output rows
    r = D.inverse(c, out=out).cpu().numpy()
    assert np.abs(r.astype(np.float64) - x).max() <= (0 if dt == torch.int32 else FLOAT_TOL)


def test_full_size_8192_int53_five_levels():
    """8192 x 8192 seeded 1/f^2 field, reversible CDF 5/3, 5 levels, the benchmark's launch
    configuration: bit-exact against the oracle and exact reconstruction."""
    x = I.field(8192, 8192, I.seed_for(1)).astype(np.int32)
    t = to_gpu(x, torch.int32)
    c = D.forward(t, "cdf53_int", 5)
    assert_bands(gpu_bands(c), O.forward(x.astype(np.int64), "cdf53_int", 5), 0, "8192 int")
    r = D.inverse(c)
    assert torch.equal(r, t)


def _full_size_float(x: np.ndarray, what: str, storage16: bool = False):
    """Forward against the oracle, inverse of the oracle's coefficients against the oracle's
    inverse, and the GPU round trip against x: every element, bound FLOAT_TOL.  With storage16,
    also the forward with bf16 and fp16 band storage against the same oracle coefficients: per
    element FLOAT_TOL + |v| 2^-8 (bf16) or |v| 2^-10 (fp16), the rounding of the stored value
    (the final LL stays fp32, bound FLOAT_TOL)."""
    H, W = x.shape
    t = to_gpu(x, torch.float32)
    want = O.forward(x.astype(np.float64), "cdf97", 5)
    c = D.forward(t, "cdf97", 5)
    assert_bands(gpu_bands(c), want, FLOAT_TOL, ("fwd", what))
    r = D.inverse(c)
    rt = (r - t).abs().max().item()
    assert rt <= FLOAT_TOL, ("roundtrip", what, rt)
    del r, c
    cc = D.alloc_coeffs(H, W, 5, "cdf97", D.DT_F32, "cuda")
    for v, wv in zip(cc.band_views(), want):
        v.copy_(torch.from_numpy(wv.astype(np.float32)))
    r2 = D.inverse(cc).cpu().numpy()
    want_x = O.inverse(want, H, W, "cdf97", 5)
    err = np.abs(r2 - want_x).max()
    assert err <= FLOAT_TOL, ("inv", what, err)
    del r2, cc, want_x
    if storage16:
        for bdt, rel in ((torch.bfloat16, 2.0 ** -8), (torch.float16, 2.0 ** -10)):
            c16 = D.forward(t, "cdf97", 5, band_dtype=bdt)
            for k, (v, w) in enumerate(zip(c16.band_views(), want)):
                assert v.dtype == (torch.float32 if k == 0 else bdt)
                if w.size == 0:
                    continue
                g = v.float().cpu().numpy().astype(np.float64)
                tol = FLOAT_TOL + (0.0 if k == 0 else rel) * np.abs(w)
                assert (np.abs(g - w) <= tol).all(), ("fwd 16-bit", what, str(bdt), k)
            del c16


def test_full_size_8192_cdf97_five_levels():
    """8192 x 8192 seeded 1/f^2 field, CDF 9/7 fp32, 5 levels (the benchmark's headline)."""
    _full_size_float(I.field(8192, 8192, I.seed_for(1)), "8192 97")


def test_full_size_16384_cdf97_five_levels():
    """16384 x 16384 field plus uniform noise in [0, 255], CDF 9/7 fp32, 5 levels (the band
    storage workload: fp32, bf16 and fp16 band storage)."""
    _full_size_float(I.field_plus_noise(16384, 16384, I.seed_for(3)), "16384 97", storage16=True)


def test_constant_image_exact_with_level_shift():
    """A constant image: the DC level shift takes the constant off exactly, so every high-pass
    band is exactly zero and LL is the constant at every level (without the shift the fp32
    constants leave high-pass values of order 1e-5 * the constant)."""
    for H, W in [(1000, 777), (64, 1)]:
        t = torch.full((H, W), 200.0, device="cuda")
        c = D.forward(t, "cdf97", min(5, D.max_levels(H, W)))
        views = c.band_views()
        assert torch.equal(views[0], torch.full_like(views[0], 200.0))
        for v in views[1:]:
            assert v.numel() == 0 or v.abs().max().item() == 0.0
        assert torch.equal(D.inverse(c), t)


def test_non_finite_sample_stays_local():
    """The level shift is sampled from a 3 x 3 grid of the image; a NaN at a sample position
    counts as 0 there, so it spoils only the coefficients that read it, as it would with no
    shift, and the rest still matches the oracle."""
    H, W = 600, 900
    x = I.field(H, W, I.seed_for(1, 7))
    x[H // 2, W // 2] = np.nan  # the centre sample
    c = D.forward(to_gpu(x, torch.float32), "cdf97", 3)
    got = gpu_bands(c)
    want = O.forward(x.astype(np.float64), "cdf97", 3)
    for g, w in zip(got, want):
        assert np.isnan(g).sum() == np.isnan(w).sum()
        ok = ~np.isnan(w)
        assert np.abs(g[ok] - w[ok]).max() <= FLOAT_TOL


def test_repeated_calls_identical():
    """Calls share nothing but the workspace: a second call gives the same bits."""
    x = I.field(1000, 777, I.seed_for(1))
    t = to_gpu(x, torch.float32)
    ws = D.new_workspace(D.workspace_bytes(1000, 777, 4, "cdf97", D.DT_F32))
    a = gpu_bands(D.forward(t, "cdf97", 4, workspace=ws))
    b = gpu_bands(D.forward(t, "cdf97", 4, workspace=ws))
    assert_bands(a, b, 0, "repeat")
    assert D.check_status(ws) == 0
