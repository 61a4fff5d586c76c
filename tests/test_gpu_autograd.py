"""Autograd through the hand-written adjoint kernels, against the fp64 oracle gradient.

Workload: the differentiation configuration's loss on a small batch,
    L = sum |high-pass coefficients| + mean((idwt2(dwt2(x)) - x)^2),  CDF 9/7, 3 levels.
The oracle gradient (pinned by finite differences in test_loss_gradient_oracle) is
W^T s + (2/N)(W^T W^-T r - r), with s the signs of the GPU's high-pass coefficients: the sign is
a decision taken once, in fp32 on the GPU, and given to both sides.  The GPU gradient is fp32;
the bound is 1e-4 relative to the gradient's size.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import autograd as A
from paper_1708_07853_gb300 import inputs as I

from test_loss_gradient_oracle import grad as oracle_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _loss(x, wavelet, lv):
    H, W = x.shape[-2:]
    c = A.dwt2(x, wavelet, lv)
    views = A.band_views(c, H, W, lv)
    xr = A.idwt2(c, H, W, wavelet, lv)
    return sum(v.abs().sum() for v in views[1:]) + ((xr - x) ** 2).mean(), c


@pytest.mark.parametrize("wavelet", ["cdf97", "cdf53"])
@pytest.mark.parametrize("shape", [(2, 3, 64, 64), (1, 1, 67, 45), (3, 40, 1)])
def test_autograd_gradient_matches_fp64_oracle(wavelet, shape):
    H, W = shape[-2:]
    lv = min(3, O.max_levels(H, W))
    n_img = int(np.prod(shape[:-2]))
    x0 = np.stack([I.field(H, W, I.seed_for(4, k), integer=False) / 255.0 for k in range(n_img)])
    x = torch.from_numpy(x0.reshape(shape).astype(np.float32)).cuda().requires_grad_(True)
    loss, c = _loss(x, wavelet, lv)
    loss.backward()
    got = x.grad.reshape(n_img, H, W).cpu().numpy().astype(np.float64)
    views = [v.reshape(n_img, *v.shape[-2:]).detach().cpu().numpy()
             for v in A.band_views(c, H, W, lv)]
    N = x.numel()
    for k in range(n_img):
        xi = x0[k].astype(np.float32).astype(np.float64)
        signs = [np.zeros(views[0][k].shape)] + [np.sign(v[k]).astype(np.float64) for v in views[1:]]
        # oracle_grad uses 2/x.size for one image; the batch mean divides by all N pixels
        g = oracle_grad(xi, signs, wavelet, lv)
        g1 = O.forward_adjoint(signs, H, W, wavelet, lv)
        want = g1 + (g - g1) * (xi.size / N)
        assert np.abs(got[k] - want).max() <= 1e-4 * max(1.0, np.abs(want).max()), k


def test_padding_stays_zero_and_layout_roundtrip():
    H, W, lv = 37, 29, 3
    x = torch.rand((2, H, W), device="cuda")
    c = A.dwt2(x, "cdf97", lv)
    views = A.band_views(c, H, W, lv)
    mask = torch.zeros_like(c, dtype=torch.bool)
    for v in A.band_views(mask, H, W, lv):
        v.fill_(True)
    assert (~mask).any()  # this layout has padding
    assert (c[~mask] == 0).all()
    xr = A.idwt2(c, H, W, "cdf97", lv)
    assert (xr - x).abs().max().item() <= 1e-3
    assert sum(v[0].numel() for v in views) == H * W
    # the gradient of the coefficients (the inverse adjoint) is zero on the padding as well,
    # on buffers that start uninitialised
    cr = c.detach().clone().requires_grad_(True)
    A.idwt2(cr, H, W, "cdf97", lv).pow(2).sum().backward()
    assert (cr.grad[~mask] == 0).all()
    assert torch.equal(A.padding_index(H, W, lv, "cuda"), torch.nonzero(~mask[0]).ravel())


def test_autograd_full_size_64x3x1024():
    """The differentiation workload at full size, as the benchmark runs it: 64 x 3 images of
    1024 x 1024 in [0, 1], 3 levels of 9/7, one forward + backward through the autograd
    Functions (batched entry points).  Three sampled images (first, middle, last) are checked
    against the fp64 oracle gradient; they get their content from the host-side generator,
    the others are drawn on the device."""
    B, C, H, W, lv = 64, 3, 1024, 1024, 3
    n_img = B * C
    picks = (0, n_img // 2, n_img - 1)
    host = {k: I.field(H, W, I.seed_for(4, k)) / 255.0 for k in picks}
    x = torch.empty((B, C, H, W), device="cuda")
    flat = x.view(-1, H, W)
    for k in range(n_img):
        if k in host:
            flat[k] = torch.from_numpy(host[k].astype(np.float32)).cuda()
        else:
            flat[k] = I.field_device(H, W, I.seed_for(4, k), "cuda") / 255.0
    x.requires_grad_(True)
    loss, c = _loss(x, "cdf97", lv)
    loss.backward()
    views = A.band_views(c, H, W, lv)
    N = x.numel()
    for k in picks:
        got = x.grad.view(-1, H, W)[k].cpu().numpy().astype(np.float64)
        xi = host[k].astype(np.float32).astype(np.float64)
        signs = [np.zeros((v.shape[-2], v.shape[-1])) for v in views[:1]] + \
                [np.sign(v.reshape(n_img, *v.shape[-2:])[k].detach().cpu().numpy()).astype(np.float64)
                 for v in views[1:]]
        g = oracle_grad(xi, signs, "cdf97", lv)
        g1 = O.forward_adjoint(signs, H, W, "cdf97", lv)
        want = g1 + (g - g1) * (xi.size / N)
        assert np.abs(got - want).max() <= 1e-4 * max(1.0, np.abs(want).max()), k
