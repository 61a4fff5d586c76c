"""GPU parity of the separable comparators (Eq. 3) against the oracle.

DWT2_SCHEME_SEP_FUSED evaluates P, P*, U, U* one after the other in a single pass: for the
integer wavelet it rounds in Eq. 3's order and is bit-exact with the oracle's Eq. 3 scheme.
DWT2_SCHEME_SEP_TWOPASS runs all row steps, then all column steps (two kernels per level): for
the integer wavelet it is bit-exact with the oracle's rows-then-columns order instead.  Float
results meet the same 1e-3 bound as the non-separable path.  DWT2_SCHEME_ADAPTED (Sec. 3's
adapted non-separable scheme, float wavelets) is compared with the oracle's adapted form and
with its Eq. 3 form, both within that bound.  DWT2_SCHEME_CONV (the separable convolution of
Eq. 4, float wavelets) filters with taps the kernel derives from its own lifting constants; the
oracle's lifting result, whose equality with the published filter banks is pinned on the CPU,
is the reference, within the same bound.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D
from paper_1708_07853_gb300 import inputs as I

from test_gpu_parity import FLOAT_TOL, assert_bands, gpu_bands, to_gpu

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (2, 3), (7, 1), (17, 16), (100, 130), (481, 480), (600, 962), (37, 1923)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


@pytest.mark.parametrize("scheme,order", [("sep_fused", "eq3"), ("sep_twopass", "rows")])
@pytest.mark.parametrize("H,W", SIZES)
def test_int53_separable(scheme, order, H, W):
    rng = np.random.default_rng(H + 31 * W)
    x = rng.integers(-(2 ** 15), 2 ** 15 + 1, (H, W)).astype(np.int32)
    for lv in sorted({1, D.max_levels(H, W)}):
        c = D.forward(to_gpu(x, torch.int32), "cdf53_int", lv, scheme=scheme)
        assert_bands(gpu_bands(c), O.forward(x.astype(np.int64), "cdf53_int", lv, order), 0,
                     (scheme, H, W, lv))


@pytest.mark.parametrize("scheme", ["sep_fused", "sep_twopass"])
@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", SIZES)
def test_float_separable(scheme, wavelet, H, W):
    rng = np.random.default_rng(H + 17 * W)
    x = rng.uniform(0, 255, (H, W)).astype(np.float32)
    for lv in sorted({1, min(5, D.max_levels(H, W))}):
        c = D.forward(to_gpu(x, torch.float32), wavelet, lv, scheme=scheme)
        assert_bands(gpu_bands(c), O.forward(x.astype(np.float64), wavelet, lv), FLOAT_TOL,
                     (scheme, wavelet, H, W, lv))


@pytest.mark.parametrize("wavelet", ["dd97", "dd137"])
@pytest.mark.parametrize("H,W", SIZES + [(1030, 1101)])
def test_dd_two_pass(wavelet, H, W):
    """The two-pass comparator of the four-tap wavelets (row kernel, then column kernel)."""
    rng = np.random.default_rng(H + 19 * W)
    x = rng.uniform(0, 255, (H, W)).astype(np.float32)
    for lv in sorted({1, min(5, D.max_levels(H, W))}):
        c = D.forward(to_gpu(x, torch.float32), wavelet, lv, scheme="sep_twopass")
        assert_bands(gpu_bands(c), O.forward(x.astype(np.float64), wavelet, lv, "rows"),
                     FLOAT_TOL, ("sep_twopass", wavelet, H, W, lv))


def test_full_size_8192_separable_matches_nonseparable():
    """At the benchmark's size every scheme computes the same transform."""
    x = I.field(8192, 8192, I.seed_for(1))
    t = to_gpu(x, torch.float32)
    ref = gpu_bands(D.forward(t, "cdf97", 5))
    for scheme in ("sep_fused", "sep_twopass"):
        assert_bands(gpu_bands(D.forward(t, "cdf97", 5, scheme=scheme)), ref, FLOAT_TOL, scheme)
    ti = to_gpu(x.astype(np.int32), torch.int32)
    refi = gpu_bands(D.forward(ti, "cdf53_int", 5))
    assert_bands(gpu_bands(D.forward(ti, "cdf53_int", 5, scheme="sep_fused")), refi, 0, "fused")


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", SIZES)
def test_float_adapted(wavelet, H, W):
    rng = np.random.default_rng(H + 23 * W)
    x = rng.uniform(0, 255, (H, W)).astype(np.float32)
    for lv in sorted({1, min(5, D.max_levels(H, W))}):
        got = gpu_bands(D.forward(to_gpu(x, torch.float32), wavelet, lv, scheme="adapted"))
        xd = x.astype(np.float64)
        assert_bands(got, O.forward(xd, wavelet, lv, "adapted"), FLOAT_TOL, (wavelet, H, W, lv))
        assert_bands(got, O.forward(xd, wavelet, lv, "eq3"), FLOAT_TOL, (wavelet, H, W, lv))


def test_adapted_full_size_and_integer_rejected():
    x = I.field(8192, 8192, I.seed_for(1))
    t = to_gpu(x, torch.float32)
    ref = gpu_bands(D.forward(t, "cdf97", 5))
    assert_bands(gpu_bands(D.forward(t, "cdf97", 5, scheme="adapted")), ref, FLOAT_TOL, "adapted")
    with pytest.raises(D.Dwt2Error):
        D.forward(to_gpu(x[:64, :64].astype(np.int32), torch.int32), "cdf53_int", 2,
                  scheme="adapted")


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("H,W", SIZES + [(2, 2), (3, 4), (5, 2), (1, 17)])
def test_float_convolution(wavelet, H, W):
    rng = np.random.default_rng(H + 29 * W)
    x = rng.uniform(0, 255, (H, W)).astype(np.float32)
    for lv in sorted({1, min(5, D.max_levels(H, W))}):
        got = gpu_bands(D.forward(to_gpu(x, torch.float32), wavelet, lv, scheme="conv"))
        assert_bands(got, O.forward(x.astype(np.float64), wavelet, lv), FLOAT_TOL,
                     (wavelet, H, W, lv))


def test_convolution_unaligned_pitch_and_full_size():
    x = I.field(8192, 8192, I.seed_for(1))
    t = to_gpu(x, torch.float32)
    ref = gpu_bands(D.forward(t, "cdf97", 5))
    assert_bands(gpu_bands(D.forward(t, "cdf97", 5, scheme="conv")), ref, FLOAT_TOL, "conv")
    small = x[:300, :517]
    want = O.forward(small.astype(np.float64), "cdf97", 4)
    got = gpu_bands(D.forward(to_gpu(small, torch.float32, pad=3), "cdf97", 4, scheme="conv"))
    assert_bands(got, want, FLOAT_TOL, "conv, plain-load path")
