"""Pins of the oracle's Deslauriers-Dubuc 9/7 and 13/7 wavelets (the interpolating wavelets,
four-tap lifting steps), against what the mathematics of the construction fixes rather than the
constants themselves:

* the predict is cubic interpolation: the high-pass bands vanish on polynomials of degree <= 3
  and not on degree 4 (four dual vanishing moments fix both predict taps);
* the update gives the low pass Ñ zeros at Nyquist (Ñ = 2 for 9/7, 4 for 13/7): it vanishes on
  (-1)^n n^k for k < Ñ and not for k = Ñ (this fixes the update taps);
* DC gain 1 (no scaling): a constant image comes back as the constant in LL, zeros elsewhere;
* the non-separable spatial steps (Eq. 5) equal the separable steps (Eq. 3), the in-step
  reflection equals lifting an extended signal, and both inverses reconstruct.
Plain numpy, CPU only.
"""
import numpy as np
import pytest

from oracle import oracle as O

DD = ["dd97", "dd137"]
N_TILDE = {"dd97": 2, "dd137": 4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


def _row_transform(x, wv):
    """One level of a 1 x N image: (low, high) of the 1-D transform."""
    b = O.forward(np.asarray(x, dtype=np.float64)[None, :], wv, 1, "eq3")
    return b[0][0], b[1][0]  # LL (1 x ceil), HL (1 x floor)


@pytest.mark.parametrize("wv", DD)
def test_high_pass_vanishes_on_cubics_not_quartics(wv):
    n = np.arange(80, dtype=np.float64)
    t = (n - 40.0) / 10.0
    for deg in range(4):
        lo, hi = _row_transform(t ** deg, wv)
        # interior odd samples: all four predict taps inside (the outer ones at distance 3)
        assert np.abs(hi[2:-2]).max() < 1e-12, (wv, deg)
    # degree 4 is not reproduced: the residual of cubic interpolation of n^4 at the midpoint of
    # the nodes -3, -1, 1, 3 (unit spacing) is (the fourth derivative / 4!) * (1)(-1)(3)(-3) = 9,
    # here times the scale 10^-4 of t = (n - 40) / 10
    lo, hi = _row_transform(t ** 4, wv)
    assert np.allclose(hi[2:-2], 9e-4, rtol=1e-9, atol=0), wv


@pytest.mark.parametrize("wv", DD)
def test_low_pass_vanishes_at_nyquist_to_its_order(wv):
    n = np.arange(96, dtype=np.float64)
    alt = np.where(n % 2 == 0, 1.0, -1.0)
    t = (n - 48.0) / 12.0
    nt = N_TILDE[wv]
    for k in range(nt):
        lo, _ = _row_transform(alt * t ** k, wv)
        assert np.abs(lo[4:-4]).max() < 1e-12, (wv, k)
    lo, _ = _row_transform(alt * t ** nt, wv)
    assert np.abs(lo[4:-4]).min() > 1e-4, wv  # order exactly Ñ


@pytest.mark.parametrize("wv", DD)
@pytest.mark.parametrize("scheme", ["eq3", "eq5"])
def test_constant_image_dc_gain_one(wv, scheme):
    H, W = 23, 30
    b = O.forward(np.full((H, W), 7.25), wv, 3, scheme)
    assert np.allclose(b[0], 7.25, atol=1e-12, rtol=0)
    for band in b[1:]:
        assert np.abs(band).max() < 1e-12


@pytest.mark.parametrize("wv", DD)
def test_two_d_high_bands_vanish_on_separable_cubics(wv):
    r = (np.arange(40.0) - 20.0) / 8.0
    c = (np.arange(44.0) - 22.0) / 8.0
    x = np.outer(r ** 3 - 2 * r, c ** 2 + c + 1.0)
    LL, HL, LH, HH = O.forward(x, wv, 1, "eq5")
    for band in (HL, LH, HH):
        assert np.abs(band[2:-2, 2:-2]).max() < 1e-10, wv


SIZES = [(1, 1), (1, 9), (9, 1), (2, 2), (3, 5), (5, 3), (7, 8), (17, 16), (33, 31), (64, 70)]


@pytest.mark.parametrize("wv", DD)
def test_nonseparable_equals_separable_and_extension(wv):
    rng = np.random.default_rng(11)
    for H, W in SIZES:
        x = rng.uniform(0, 255, (H, W))
        L = O.max_levels(H, W)
        a = O.forward(x, wv, L, "eq3")
        b = O.forward(x, wv, L, "eq5")
        c = O.forward(x, wv, L, "eq3", extension_form=True)
        for p, q, s in zip(a, b, c):
            if p.size:
                assert np.abs(p - q).max() <= 1e-10, (wv, H, W)
                assert np.array_equal(p, s), (wv, H, W)


@pytest.mark.parametrize("wv", DD)
@pytest.mark.parametrize("scheme", ["eq3", "eq5"])
def test_perfect_reconstruction_dd(wv, scheme):
    rng = np.random.default_rng(12)
    for H, W in SIZES:
        x = rng.uniform(0, 255, (H, W))
        L = O.max_levels(H, W)
        r = O.inverse(O.forward(x, wv, L, scheme), H, W, wv, L, scheme)
        assert np.abs(r - x).max() <= 1e-9, (wv, scheme, H, W)


def test_dd_differ_from_cdf53_only_by_the_outer_taps():
    """The 9/7 and 13/7 share the predict; they differ in the update only."""
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 255, (20, 24))
    a = O.forward(x, "dd97", 1, "eq3")
    b = O.forward(x, "dd137", 1, "eq3")
    # same predict: the HH band of one level depends on the predict alone
    assert np.array_equal(a[3], b[3])
    assert np.abs(a[0] - b[0]).max() > 1e-3
