"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a published filter bank (golden taps), a value
derived by hand (golden files), a closed form (constant / ramp / polynomial inputs), an
algebraic identity of the paper (Eq. 3 = Eq. 5 in exact arithmetic; Sec. 3 on which component
each fused step writes), or linear algebra (a dense matrix and its literal transpose).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17]


def _ints(s):
    return [int(t) for t in s.split()]


# --------------------------------------------------------------------------- golden: integer

def test_int53_1d_hand_vectors():
    for line in open(os.path.join(GOLD, "cdf53_int_1d.txt")):
        if line.startswith("#") or not line.strip():
            continue
        x, L, H = (_ints(p) for p in line.split("|"))
        b = O.forward(np.array([x]), "cdf53_int", 1)
        assert b[0].ravel().tolist() == L and b[1].ravel().tolist() == H, line
        # the same vector as a column (vertical steps) gives L in LL and H in LH
        b = O.forward(np.array([x]).T, "cdf53_int", 1)
        assert b[0].ravel().tolist() == L and b[2].ravel().tolist() == H, line


def test_int53_2d_hand_example_fixes_step_order():
    rows = {}
    for line in open(os.path.join(GOLD, "cdf53_int_2d_4x4.txt")):
        if line.startswith("#") or ":" not in line:
            continue
        k, v = line.split(":", 1)
        rows[k.strip()] = np.array([_ints(r) for r in v.split(";")])
    x = rows["input"]
    for scheme in ("eq3", "eq5"):
        LL, HL, LH, HH = O.forward(x, "cdf53_int", 1, scheme)
        for name, got in (("LL", LL), ("HL", HL), ("LH", LH), ("HH", HH)):
            assert (got == rows[name]).all(), (scheme, name, got)
    # rows-first rounding order differs on this example (Sec. 2's free interleaving is exact
    # arithmetic only), so the fixture distinguishes the order
    LLr = O.forward(x, "cdf53_int", 1, "rows")[0]
    assert not (LLr == rows["LL"]).all()


# ------------------------------------------------------- golden: published filter bank (Eq. 4)

def _taps():
    t = {}
    for line in open(os.path.join(GOLD, "analysis_taps.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, vals = line.split(":")
        wv, ch, sc = head.split()
        t[(wv, ch)] = np.array([float(v) for v in vals.split()]) * float(sc)
    return t


TAPS = _taps()


def _analysis_axis(x, lo, hi, axis):
    """Filter-bank analysis along one axis (convolve, then subsample), on the signal extended by
    numpy's 'reflect' padding (whole-sample symmetric, repeated for short signals)."""
    n = x.shape[axis]
    if n == 1:
        return x.copy(), np.take(x, np.arange(0), axis=axis)
    E = 8
    pad = [(E, E) if a == axis else (0, 0) for a in range(x.ndim)]
    xe = np.pad(x, pad, mode="reflect")
    kl, kh = (len(lo) - 1) // 2, (len(hi) - 1) // 2
    nL, nH = (n + 1) // 2, n // 2
    L = sum(lo[k + kl] * np.take(xe, E + 2 * np.arange(nL) + k, axis=axis)
            for k in range(-kl, kl + 1))
    H = sum(hi[k + kh] * np.take(xe, E + 2 * np.arange(nH) + 1 + k, axis=axis)
            for k in range(-kh, kh + 1))
    return L, H


def _brute_force(x, wavelet, levels):
    """Separable convolution scheme (Eq. 4): all horizontal filtering in one step, then all
    vertical, recursing on LL; returns the band list."""
    lo, hi = TAPS[(wavelet, "low")], TAPS[(wavelet, "high")]
    out = []
    cur = x
    for _ in range(levels):
        Lr, Hr = _analysis_axis(cur, lo, hi, 1)
        LL, LH = _analysis_axis(Lr, lo, hi, 0)
        HL, HH = _analysis_axis(Hr, lo, hi, 0)
        out = [HL, LH, HH] + out
        cur = LL
    return [cur] + out


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_float_matches_published_filter_bank_one_level(wavelet):
    rng = np.random.default_rng(11)
    for H in SIZES:
        for W in SIZES:
            x = rng.standard_normal((H, W))
            got = O.forward(x, wavelet, 1)
            want = _brute_force(x, wavelet, 1)
            for g, w in zip(got, want):
                assert g.shape == w.shape
                if g.size:
                    assert np.abs(g - w).max() < 1e-12, (wavelet, H, W)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_float_matches_published_filter_bank_all_levels(wavelet):
    rng = np.random.default_rng(12)
    for H, W in [(17, 17), (16, 13), (1, 17), (9, 1), (33, 20), (64, 48), (5, 40)]:
        for lv in range(1, O.max_levels(H, W) + 1):
            x = rng.uniform(0, 255, (H, W))
            got = O.forward(x, wavelet, lv)
            want = _brute_force(x, wavelet, lv)
            for g, w in zip(got, want):
                if g.size:
                    assert np.abs(g - w).max() < 1e-10, (wavelet, H, W, lv)


# ------------------------------------------------------------------ reconstruction and schemes

@pytest.mark.parametrize("scheme", ["eq3", "eq5"])
def test_perfect_reconstruction_integer_bit_exact(scheme):
    rng = np.random.default_rng(21)
    for H, W in [(1, 1), (1, 7), (6, 1), (2, 2), (3, 3), (9, 10), (17, 16), (31, 33), (64, 70)]:
        for lv in range(1, O.max_levels(H, W) + 1):
            x = rng.integers(-(2 ** 15), 2 ** 15 + 1, (H, W))
            b = O.forward(x, "cdf53_int", lv, scheme)
            assert (O.inverse(b, H, W, "cdf53_int", lv, scheme) == x).all(), (H, W, lv)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
@pytest.mark.parametrize("scheme", ["eq3", "eq5"])
def test_perfect_reconstruction_float(wavelet, scheme):
    rng = np.random.default_rng(22)
    for H, W in [(1, 1), (1, 7), (6, 1), (2, 2), (3, 3), (9, 10), (17, 16), (31, 33), (64, 70)]:
        for lv in range(1, O.max_levels(H, W) + 1):
            x = rng.uniform(0, 255, (H, W))
            b = O.forward(x, wavelet, lv, scheme)
            r = O.inverse(b, H, W, wavelet, lv, scheme)
            assert np.abs(r - x).max() < 1e-10, (H, W, lv)


def test_nonseparable_equals_separable():
    """Eq. 5 multiplies out Eq. 3's matrices, so both give the same coefficients: bit-exact for
    the integer wavelet (the fused steps keep Eq. 3's floors), within fp64 rounding for float."""
    rng = np.random.default_rng(31)
    for H in SIZES:
        for W in SIZES:
            lv = O.max_levels(H, W)
            x = rng.integers(-300, 300, (H, W))
            a = O.forward(x, "cdf53_int", lv, "eq3")
            b = O.forward(x, "cdf53_int", lv, "eq5")
            assert all((p == q).all() for p, q in zip(a, b)), (H, W)
            xf = rng.standard_normal((H, W))
            for wv in ("cdf53", "cdf97"):
                a = O.forward(xf, wv, lv, "eq3")
                b = O.forward(xf, wv, lv, "eq5")
                assert max((np.abs(p - q).max() if p.size else 0) for p, q in zip(a, b)) < 1e-12


def test_adapted_scheme_equals_separable():
    """Sec. 3's adapted scheme splits P = P0 + P1, U = U0 + U1; each spatial step factors into a
    local step with the constants and a fused step with the rest, so the level is the same
    linear map as Eq. 3's: within fp64 rounding, every size (odd, length 1) and level count."""
    rng = np.random.default_rng(32)
    for H in SIZES:
        for W in SIZES:
            lv = O.max_levels(H, W)
            xf = rng.standard_normal((H, W))
            for wv in ("cdf53", "cdf97"):
                a = O.forward(xf, wv, lv, "eq3")
                b = O.forward(xf, wv, lv, "adapted")
                assert max((np.abs(p - q).max() if p.size else 0) for p, q in zip(a, b)) < 1e-12
    with pytest.raises(ValueError):  # no integer form: the split would change the floors
        O.forward(rng.integers(0, 9, (8, 8)), "cdf53_int", 1, "adapted")


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_adapted_local_steps_read_no_neighbours(wavelet):
    """Sec. 3: the detached constant parts never access results of other quads.  Perturbing one
    quad before a local step (predict or update, every lifting pair) changes that quad only;
    before a fused step it reaches the neighbours."""
    rng = np.random.default_rng(33)
    H, W = 14, 18
    ner, ndr, nec, ndc = 7, 7, 9, 9
    shapes = [(ner, nec), (ner, ndc), (ndr, nec), (ndr, ndc)]
    nsteps = 8 if wavelet == "cdf97" else 4
    for k in range(nsteps):
        base = [rng.standard_normal(s) for s in shapes]
        pert = [p.copy() for p in base]
        for p in pert:
            p[3, 4] += 1.0
        d = [q - p for p, q in zip(O.adapted_apply(base, H, W, wavelet, k, k + 1),
                                   O.adapted_apply(pert, H, W, wavelet, k, k + 1))]
        changed_elsewhere = max(float(np.abs(x).sum() - abs(x[3, 4])) for x in d)
        if k % 2 == 0:  # local step
            assert changed_elsewhere < 1e-12, (k, changed_elsewhere)
        else:           # fused step: the perturbation reaches a neighbour
            assert changed_elsewhere > 1e-6, k


def test_extension_form_equals_in_step_reflection():
    """Whole-sample symmetric extension defined on the signal (extend, lift, crop) equals the
    reflection rule applied inside each lifting step."""
    rng = np.random.default_rng(32)
    for H in SIZES:
        for W in (1, 2, 3, 5, 8, 13, 16, 17):
            lv = O.max_levels(H, W)
            x = rng.integers(-300, 300, (H, W))
            a = O.forward(x, "cdf53_int", lv, "eq3", False)
            b = O.forward(x, "cdf53_int", lv, "eq3", True)
            assert all((p == q).all() for p, q in zip(a, b)), (H, W)
            xf = rng.standard_normal((H, W))
            for wv in ("cdf53", "cdf97"):
                a = O.forward(xf, wv, lv, "eq3", False)
                b = O.forward(xf, wv, lv, "eq3", True)
                assert max((np.abs(p - q).max() if p.size else 0) for p, q in zip(a, b)) < 1e-12


def test_float_step_order_is_free():
    """Sec. 2: horizontal and vertical steps may be interleaved arbitrarily (exact arithmetic)."""
    rng = np.random.default_rng(33)
    for H, W in [(9, 10), (17, 16), (32, 31)]:
        x = rng.standard_normal((H, W))
        for wv in ("cdf53", "cdf97"):
            ref = O.forward(x, wv, 2, "eq3")
            for s in ("rows", "cols"):
                got = O.forward(x, wv, 2, s)
                assert max(np.abs(p - q).max() for p, q in zip(ref, got)) < 1e-12


def test_integer_step_order_matters():
    rng = np.random.default_rng(34)
    x = rng.integers(0, 256, (9, 10))
    a = O.forward(x, "cdf53_int", 1, "eq3")
    b = O.forward(x, "cdf53_int", 1, "rows")
    assert any((p != q).any() for p, q in zip(a, b))


def test_fused_steps_write_the_components_sec3_names():
    """Sec. 3: the spatial predict is responsible for HH (and leaves LL alone); the spatial
    update is responsible for LL (and leaves HH alone)."""
    rng = np.random.default_rng(35)
    x = rng.standard_normal((10, 11))
    for wv, npairs in (("cdf53", 1), ("cdf97", 2)):
        prev = O.nonsep_steps(x, wv, 0)
        for k in range(2 * npairs):
            cur = O.nonsep_steps(x, wv, k + 1)
            if k % 2 == 0:  # predict
                assert (cur[0] == prev[0]).all()
                assert not np.allclose(cur[3], prev[3])
            else:  # update
                assert (cur[3] == prev[3]).all()
                assert not np.allclose(cur[0], prev[0])
            prev = cur


# ------------------------------------------------------------------------ closed-form inputs

@pytest.mark.parametrize("wavelet", ["cdf53_int", "cdf53", "cdf97"])
def test_constant_input(wavelet):
    """A constant has no high-pass content; the low-pass DC gain is 1 at every level."""
    for H, W in [(1, 5), (7, 1), (8, 8), (13, 9), (33, 64)]:
        lv = O.max_levels(H, W)
        c = 77
        x = np.full((H, W), c)
        b = O.forward(x, wavelet, lv)
        tol = 0 if wavelet != "cdf97" else 1e-12 * c
        assert np.abs(b[0] - c).max() <= tol
        for band in b[1:]:
            if band.size:
                assert np.abs(band).max() <= tol


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_dc_level_shift_is_exact(wavelet):
    """The float kernels transform x - c and add c back to LL_J (a DC level shift that keeps
    their fp32 intermediates small).  By linearity and the constant-input facts above (LL gain
    1, zero high-pass) that is the same transform: W(x - c) + c e_LL = W(x), and the inverse
    of the bands with LL_J - c, plus c, is the inverse of the bands.  Checked on odd sizes,
    length-1 axes and every level count, where the symmetric extension meets the boundary."""
    rng = np.random.default_rng(17)
    for H, W in [(1, 9), (6, 1), (13, 9), (33, 64), (40, 17)]:
        x = rng.uniform(0, 255, (H, W))
        for lv in range(1, O.max_levels(H, W) + 1):
            c = 131.0
            want = O.forward(x, wavelet, lv)
            got = O.forward(x - c, wavelet, lv)
            got[0] = got[0] + c
            for g, w in zip(got, want):
                assert np.abs(g - w).max(initial=0) <= 1e-12 * 255, (H, W, lv)
            shifted = [want[0] - c] + list(want[1:])
            r = O.inverse(shifted, H, W, wavelet, lv) + c
            assert np.abs(r - x).max() <= 1e-12 * 255, (H, W, lv)


def _h1d(x, wavelet):
    return O.forward(np.asarray(x)[None, :], wavelet, 1)[1].ravel()


def test_ramp_and_polynomials():
    """Vanishing moments: CDF 5/3 high-pass kills linear signals (2 moments), CDF 9/7 kills
    up to cubics (4 moments), except where the symmetric extension breaks the polynomial."""
    r17, r16 = np.arange(17.0), np.arange(16.0)
    h = _h1d(r17, "cdf53")
    assert np.abs(h).max() == 0  # odd length: the reflection at the end is still linear
    h = _h1d(r16, "cdf53")
    assert np.abs(h[:-1]).max() == 0 and h[-1] == 1.0  # the last detail sees x[16] = x[14]
    hi = _h1d(np.arange(16), "cdf53_int")
    assert (hi[:-1] == 0).all() and hi[-1] == 1
    h = _h1d(r17, "cdf97")
    assert np.abs(h[1:-1]).max() < 1e-12
    assert abs(h[0] - 0.125) < 1e-12 and abs(h[-1] + 0.125) < 1e-12
    for p in (2, 3):
        h = _h1d(r17 ** p, "cdf97")
        assert np.abs(h[1:-1]).max() < 1e-9 * 17 ** p
        assert abs(h[-1]) > 1e-3  # the reflection about sample 16 is not the polynomial
        # about sample 0 the reflection of n^2 is n^2 again (even), that of n^3 is not
        assert (abs(h[0]) < 1e-9) if p == 2 else (abs(h[0]) > 1e-3)
    # 2-D: a plane ramp x[r][c] = r + 2c has zero HL/LH/HH away from the last row/column
    H, W = 15, 17
    x = np.add.outer(np.arange(H), 2 * np.arange(W)).astype(float)
    LL, HL, LH, HH = O.forward(x, "cdf53", 1)
    assert np.abs(HL).max() == 0 and np.abs(LH).max() == 0 and np.abs(HH).max() == 0


def test_cdf97_gains():
    """Normalisation of the 9/7: low-pass DC gain 1, high-pass Nyquist gain 1."""
    alt = np.array([(-1.0) ** k for k in range(32)])
    b = O.forward(alt[None, :], "cdf97", 1)
    assert np.abs(b[0][0, 2:-2]).max() < 1e-12
    assert np.abs(b[1][0, 2:-2] + 1.0).max() < 1e-12


def test_integer_close_to_float_with_derived_bound():
    """The integer steps differ from the float steps by the rounding of each floor (at most 1/2
    per step).  Propagating that through P, P*, U, U* from an exact integer input bounds one
    level by LL 2.125, HL 1.75, LH 1.75, HH 1.5; a second level adds the first level's LL error
    times the filter's l1 gain (5/3 low 1.5, high 2 per axis)."""
    rng = np.random.default_rng(41)
    b1 = {"LL": 2.125, "HL": 1.75, "LH": 1.75, "HH": 1.5}
    b2 = {"LL": 2.25 * 2.125 + 2.125, "HL": 3 * 2.125 + 1.75, "LH": 3 * 2.125 + 1.75,
          "HH": 4 * 2.125 + 1.5}
    for _ in range(10):
        H, W = rng.integers(20, 70, 2)
        x = rng.integers(0, 256, (H, W))
        for lv, bound in ((1, b1), (2, b2)):
            bi = O.forward(x, "cdf53_int", lv)
            bf = O.forward(x.astype(float), "cdf53", lv)
            for (kind, j, _, _), p, q in zip(O.band_shapes(H, W, lv), bi, bf):
                if p.size:
                    lim = bound[kind] if (lv == 1 or j == 2 or kind == "LL") else b1[kind]
                    assert np.abs(p - q).max() <= lim, (kind, j, lv)


# --------------------------------------------------------------------------------- adjoints

def _dense(fn, n_in):
    cols = []
    for i in range(n_in):
        e = np.zeros(n_in)
        e[i] = 1.0
        cols.append(fn(e))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_adjoint_is_literal_transpose(wavelet):
    for H, W in [(1, 2), (2, 1), (2, 2), (3, 4), (5, 3), (6, 7), (8, 8), (9, 5)]:
        for lv in range(1, O.max_levels(H, W) + 1):
            n = H * W

            def fwd(v):
                return O.join_bands(O.forward(v.reshape(H, W), wavelet, lv))

            def inv(v):
                return O.inverse(O.split_bands(v, H, W, lv), H, W, wavelet, lv).ravel()

            def fadj(v):
                return O.forward_adjoint(O.split_bands(v, H, W, lv), H, W, wavelet, lv).ravel()

            def iadj(v):
                return O.join_bands(O.inverse_adjoint(v.reshape(H, W), wavelet, lv))

            Wm, Wi = _dense(fwd, n), _dense(inv, n)
            assert np.abs(_dense(fadj, n) - Wm.T).max() < 1e-12, (H, W, lv)
            assert np.abs(_dense(iadj, n) - Wi.T).max() < 1e-12, (H, W, lv)
            assert np.abs(Wi @ Wm - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_adjoint_dot_product(wavelet):
    rng = np.random.default_rng(51)
    for H, W, lv in [(64, 48, 3), (33, 17, 4), (100, 1, 2), (31, 64, 5)]:
        x = rng.standard_normal((H, W))
        y = [rng.standard_normal(b.shape) for b in O.forward(x, wavelet, lv)]
        lhs = sum((p * q).sum() for p, q in zip(O.forward(x, wavelet, lv), y))
        rhs = (x * O.forward_adjoint(y, H, W, wavelet, lv)).sum()
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)) * H * W
        lhs = (O.inverse(y, H, W, wavelet, lv) * x).sum()
        rhs = sum((p * q).sum() for p, q in zip(y, O.inverse_adjoint(x, wavelet, lv)))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs)) * H * W


# ----------------------------------------------------------------------------- layout, args

def test_threads_do_not_change_results():
    """The multi-threaded oracle (the CPU baseline over all host cores) only shares out the
    independent lines of each 1-D step among threads: every value is the same bits."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 255, (301, 517))
    xi = rng.integers(-(2 ** 15), 2 ** 15, (301, 517))
    try:
        O.set_threads(4)
        many = [O.forward(x, "cdf97", 4), O.forward(xi, "cdf53_int", 4),
                O.forward_adjoint(O.forward(x, "cdf97", 4), 301, 517, "cdf97", 4)]
        many.append(O.inverse(many[0], 301, 517, "cdf97", 4))
    finally:
        O.set_threads(1)
    one = [O.forward(x, "cdf97", 4), O.forward(xi, "cdf53_int", 4),
           O.forward_adjoint(O.forward(x, "cdf97", 4), 301, 517, "cdf97", 4)]
    one.append(O.inverse(one[0], 301, 517, "cdf97", 4))
    for a, b in zip(many, one):
        for u, v in zip(a if isinstance(a, list) else [a], b if isinstance(b, list) else [b]):
            assert np.array_equal(u, v)


def test_layout_and_level_limits():
    assert O.max_levels(1, 1) == 1
    assert O.max_levels(8, 8) == 3
    assert O.max_levels(9, 2) == 4
    assert O.max_levels(8192, 8192) == 13
    for H, W in [(1, 1), (8, 8), (9, 2), (63, 4096)]:
        for lv in range(1, O.max_levels(H, W) + 1):
            shapes = O.band_shapes(H, W, lv)
            assert sum(h * w for *_, h, w in shapes) == H * W
    with pytest.raises(ValueError):
        O.forward(np.zeros((8, 8)), "cdf53", 4)
    with pytest.raises(ValueError):
        O.forward(np.zeros((8, 8)), "cdf53", 0)
