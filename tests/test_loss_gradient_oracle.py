"""The fp64 oracle gradient of the differentiation workload's loss, pinned by central finite
differences (CPU only).

    L(x) = sum over every high-pass band (HL, LH, HH of all levels) of |c|
           + mean((W^-1 W x - x)^2),          c = W x  (CDF 9/7, 3 levels)
    dL/dx = W^T s + (2/N) (W^T W^-T r - r),    s = sign(c) on high-pass bands, 0 on LL_J,
                                               r = W^-1 W x - x,  N = number of pixels.
The L1 term has a kink where a coefficient is 0; coordinates whose step could cross it are
skipped (sign(0) = 0 is the convention of both gradients).
"""
import numpy as np

from oracle import oracle as O


def loss(x, wavelet="cdf97", lv=3):
    H, W = x.shape
    c = O.forward(x, wavelet, lv)
    r = O.inverse(c, H, W, wavelet, lv) - x
    return sum(np.abs(b).sum() for b in c[1:]) + (r * r).mean()


def grad(x, signs, wavelet="cdf97", lv=3):
    H, W = x.shape
    c = O.forward(x, wavelet, lv)
    r = O.inverse(c, H, W, wavelet, lv) - x
    g1 = O.forward_adjoint(signs, H, W, wavelet, lv)
    wtr = O.forward_adjoint(O.inverse_adjoint(r, wavelet, lv), H, W, wavelet, lv)
    return g1 + (2.0 / x.size) * (wtr - r)


def high_pass_signs(c):
    return [np.zeros_like(c[0])] + [np.sign(b) for b in c[1:]]


def test_loss_gradient_matches_central_differences_64x64():
    rng = np.random.default_rng(77)
    H = W = 64
    x = rng.uniform(0, 1, (H, W))
    c = O.forward(x, "cdf97", 3)
    g = grad(x, high_pass_signs(c))
    eps = 1e-6
    # a coefficient can move by at most eps * (l1 norm of a column of W) <= eps * 4 per step
    cmin = min(np.abs(b).min() for b in c[1:] if b.size)
    coords = [(i, j) for i in range(H) for j in range(W)]
    pick = rng.choice(len(coords), 400, replace=False)
    checked = 0
    for k in pick:
        i, j = coords[k]
        if cmin < 10 * eps:  # a kink within reach of the step: skip this input entirely
            break
        xp, xm = x.copy(), x.copy()
        xp[i, j] += eps
        xm[i, j] -= eps
        fd = (loss(xp) - loss(xm)) / (2 * eps)
        assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(g[i, j])) + 1e-7, (i, j, fd, g[i, j])
        checked += 1
    assert checked == len(pick)


def test_reconstruction_term_gradient_is_tiny():
    """Perfect reconstruction makes the MSE term's gradient vanish up to fp64 rounding."""
    rng = np.random.default_rng(78)
    x = rng.uniform(0, 1, (40, 52))
    zero = [np.zeros(b.shape) for b in O.forward(x, "cdf97", 3)]
    assert np.abs(grad(x, zero)).max() < 1e-12
