"""Batched plans (one persistent launch for every level of every image) against the
single-image entry points and the oracle.

A plan computes each output with the same lifting arithmetic as the single-image kernels; only
the tiling (rows per tile, which CTA runs which tile) differs, and every tile recomputes its halo
from the same inputs.  So each image's result must equal the single-image result bit for bit,
for every wavelet and storage type; a sample of images is also checked against the oracle
(integer: exact; float: the 1e-3 bound of the other tests).
"""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1708_07853_gb300 import dwt2 as D
from paper_1708_07853_gb300 import inputs as I

from test_gpu_parity import FLOAT_TOL, assert_bands, gpu_bands

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1708_07853_gb300 import build as B
    B.build()


def _images(sizes, dtype, seed, pad_odd=True):
    g = torch.Generator(device="cuda").manual_seed(seed)
    out = []
    for k, (h, w) in enumerate(sizes):
        # every other image gets an unaligned pitch (plain-load path inside the plan)
        pad = 1 if (pad_odd and k % 2) else 0
        t = torch.rand((h, w + pad), generator=g, device="cuda") * 255.0
        t = t[:, :w]
        out.append(t.round().to(torch.int32) if dtype == torch.int32 else t.to(dtype))
    return out


def _same(a: D.Coeffs, b: D.Coeffs):
    for x, y in zip(a.band_views(), b.band_views()):
        assert torch.equal(x, y)


SIZES = I.batch_sizes(20, I.seed_for(3, 1), lo=17, hi=700) + [(63, 1500), (1023, 65), (17, 17)]


@pytest.mark.parametrize("wavelet,dtype,bdt", [("cdf53_int", torch.int32, D.DT_I32),
                                               ("cdf53", torch.float32, D.DT_F32),
                                               ("cdf97", torch.float32, D.DT_F32),
                                               ("cdf97", torch.float32, D.DT_BF16),
                                               ("cdf53", torch.float32, D.DT_F16),
                                               ("dd97", torch.float32, D.DT_F32),
                                               ("dd137", torch.float32, D.DT_F32),
                                               ("dd137", torch.float32, D.DT_BF16)])
def test_forward_plan_equals_single_image(wavelet, dtype, bdt):
    imgs = _images(SIZES, dtype, 11)
    plan, coeffs = D.plan_forward(imgs, wavelet, 4, band_dtype=bdt)
    plan.run()
    torch.cuda.synchronize()
    for x, c in zip(imgs, coeffs):
        _same(c, D.forward(x, wavelet, 4, band_dtype=bdt))
    for k in (0, 5, len(imgs) - 1):  # oracle sample
        x = imgs[k].cpu().numpy()
        want = O.forward(x.astype(np.int64 if dtype == torch.int32 else np.float64), wavelet, 4)
        got = gpu_bands(coeffs[k])
        for g, w in zip(got, want):
            if w.size == 0:
                continue
            if dtype == torch.int32:
                assert (g == w).all()
            else:
                rel = 0.0 if bdt == D.DT_F32 else 2.0 ** -8
                assert (np.abs(g.astype(np.float64) - w) <= FLOAT_TOL + rel * np.abs(w)).all()
    assert D.check_status(plan.workspace) == 0


@pytest.mark.parametrize("wavelet,dtype", [("cdf53_int", torch.int32), ("cdf97", torch.float32),
                                           ("dd97", torch.float32), ("dd137", torch.float32)])
def test_inverse_plan_equals_single_image(wavelet, dtype):
    imgs = _images(SIZES, dtype, 12)
    coeffs = [D.forward(x, wavelet, 4) for x in imgs]
    outs = [torch.empty_like(x) for x in imgs]
    plan = D.Plan(outs, coeffs, wavelet, 4, "inverse")
    plan.run()
    torch.cuda.synchronize()
    for o, c, x in zip(outs, coeffs, imgs):
        assert torch.equal(o, D.inverse(c))
        if dtype == torch.int32:
            assert torch.equal(o, x)


@pytest.mark.parametrize("wavelet", ["cdf53", "cdf97"])
def test_adjoint_plans_equal_single_image(wavelet):
    g = torch.Generator(device="cuda").manual_seed(13)
    sizes = SIZES[:10]
    gimgs = [torch.randn((h, w), generator=g, device="cuda") for h, w in sizes]
    # W^-T: image gradient -> band gradients
    outs = [D.alloc_coeffs(h, w, 3, wavelet, D.DT_F32, "cuda") for h, w in sizes]
    plan = D.Plan(gimgs, outs, wavelet, 3, "inverse_adjoint", D.DT_F32)
    plan.run()
    torch.cuda.synchronize()
    for x, c in zip(gimgs, outs):
        _same(c, D.inverse_adjoint(x, wavelet, 3))
    # W^T: band gradients -> image gradient
    res = [torch.empty_like(x) for x in gimgs]
    plan2 = D.Plan(res, outs, wavelet, 3, "forward_adjoint", D.DT_F32)
    plan2.run()
    torch.cuda.synchronize()
    for r, c in zip(res, outs):
        assert torch.equal(r, D.forward_adjoint(c))


def test_graph_replay_is_deterministic():
    imgs = _images(SIZES[:8], torch.float32, 14)
    plan, coeffs = D.plan_forward(imgs, "cdf97", 4)
    plan.run()
    first = [c.buffer.clone() for c in coeffs]
    for _ in range(3):
        plan.run()
    torch.cuda.synchronize()
    for a, c in zip(first, coeffs):
        assert torch.equal(a, c.buffer)


def test_tiny_images():
    sizes = [(1, 1), (1, 2), (2, 1), (3, 5), (7, 4), (2, 9), (9, 2), (4, 4)]
    for lv in (1, 2):
        ok = [s for s in sizes if D.max_levels(*s) >= lv]
        imgs = _images(ok, torch.int32, 15, pad_odd=False)
        plan, coeffs = D.plan_forward(imgs, "cdf53_int", lv)
        plan.run()
        torch.cuda.synchronize()
        for x, c in zip(imgs, coeffs):
            want = O.forward(x.cpu().numpy().astype(np.int64), "cdf53_int", lv)
            for gv, w in zip(c.band_views(), want):
                assert np.array_equal(gv.cpu().numpy(), w)


def test_autotune_writes_and_reuses_cache(tmp_path):
    cache = str(tmp_path / "tune.txt")
    imgs = _images(SIZES[:6], torch.float32, 16)
    plan, coeffs = D.plan_forward(imgs, "cdf97", 3, tune_cache=cache)
    info = plan.info()
    lines = open(cache).read().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == 1
    plan2, _ = D.plan_forward(imgs, "cdf97", 3, tune_cache=cache)
    assert plan2.info() == info
    assert len([ln for ln in open(cache).read().split("\n") if ln.strip()]) == 1
    plan2.run()
    torch.cuda.synchronize()
    for x, c in zip(imgs, plan2.coeffs):
        _same(c, D.forward(x, "cdf97", 3))


def test_log_uniform_batch_64():
    """64 images, sides log-uniform on [63, 1024] (the batching workload's distribution,
    scaled down), reversible 5/3 and CDF 9/7, 4 levels."""
    sizes = I.batch_sizes(64, I.seed_for(3, 2), lo=63, hi=1024)
    for wavelet, dtype in (("cdf53_int", torch.int32), ("cdf97", torch.float32)):
        imgs = _images(sizes, dtype, 17)
        plan, coeffs = D.plan_forward(imgs, wavelet, 4)
        plan.run()
        torch.cuda.synchronize()
        for x, c in zip(imgs, coeffs):
            _same(c, D.forward(x, wavelet, 4))


@pytest.mark.parametrize("wavelet,dtype", [("cdf53_int", torch.int32), ("cdf97", torch.float32),
                                           ("dd137", torch.float32)])
def test_large_image_plan_many_row_blocks(wavelet, dtype):
    """One 4100 x 3000 image (plus two small ones), 5 levels: many tiles per level and many
    CTAs waiting on each level's completion counter, forward and inverse, bit for bit against
    the single-image calls."""
    imgs = _images([(4100, 3000), (300, 517), (63, 64)], dtype, 18)
    plan, coeffs = D.plan_forward(imgs, wavelet, 5)
    plan.run()
    torch.cuda.synchronize()
    assert D.check_status(plan.workspace) == 0
    for x, c in zip(imgs, coeffs):
        _same(c, D.forward(x, wavelet, 5))
    outs = [torch.empty_like(x) for x in imgs]
    inv = D.Plan(outs, coeffs, wavelet, 5, "inverse")
    inv.run()
    torch.cuda.synchronize()
    assert D.check_status(inv.workspace) == 0
    for o, c in zip(outs, coeffs):
        assert torch.equal(o, D.inverse(c))


@pytest.mark.parametrize("wavelet", ["cdf97", "dd137"])
@pytest.mark.parametrize("bdt", [D.DT_BF16, D.DT_F16])
def test_inverse_plan_16bit_bands(bdt, wavelet):
    """Inverse plans read 16-bit detail bands (fp32 LL) and reconstruct fp32 images bit for bit
    as the single-image inverse does."""
    imgs = _images(SIZES[:12], torch.float32, 19)
    plan, coeffs = D.plan_forward(imgs, wavelet, 4, band_dtype=bdt)
    plan.run()
    outs = [torch.empty_like(x) for x in imgs]
    inv = D.Plan(outs, coeffs, wavelet, 4, "inverse", bdt)
    inv.run()
    torch.cuda.synchronize()
    assert D.check_status(inv.workspace) == 0
    for o, c in zip(outs, coeffs):
        assert torch.equal(o, D.inverse(c, img_dtype=torch.float32))


def test_full_batch_512_uneven_against_oracle(tmp_path):
    """The batching workload at full size, in the benchmark's launch configuration: the 512
    seeded sizes (each side log-uniform on [63, 4096]), 4 levels, one plan autotuned into a fresh
    tune cache.  Every image equals the single-image calls bit for bit; sampled images (the
    largest, the smallest, the median, the largest whose rows TMA can address and three with
    widths that are not a multiple of 4, which take the plain-load path) are checked against the
    oracle: bit-exact for the reversible 5/3,
    within the fp32 bound for 9/7.  The sampled images get their content from the host-side
    generator (the oracle's input); the others are drawn on the device."""
    sizes = I.batch_sizes(512, I.seed_for(3))
    area = np.array([h * w for h, w in sizes])
    order = np.argsort(area, kind="stable")
    odd = [k for k, (h, w) in enumerate(sizes) if w % 4][::97][:3]
    aligned = max((k for k, (h, w) in enumerate(sizes) if w % 4 == 0), key=lambda k: area[k])
    picks = sorted({int(order[-1]), int(order[0]), int(order[len(order) // 2]), aligned, *odd})
    host = {k: I.field(*sizes[k], I.seed_for(3, k)) for k in picks}
    for wavelet, dtype in (("cdf53_int", torch.int32), ("cdf97", torch.float32)):
        imgs = [torch.from_numpy(host[k]).cuda().to(dtype) if k in host else
                I.field_device(h, w, I.seed_for(3, k), "cuda").to(dtype)
                for k, (h, w) in enumerate(sizes)]
        plan, coeffs = D.plan_forward(imgs, wavelet, 4,
                                      tune_cache=str(tmp_path / f"tune_{wavelet}.txt"))
        plan.run()
        torch.cuda.synchronize()
        assert D.check_status(plan.workspace) == 0
        for x, c in zip(imgs, coeffs):
            _same(c, D.forward(x, wavelet, 4))
        for k in picks:
            x = host[k]
            if wavelet == "cdf53_int":
                want = O.forward(x.astype(np.int64), wavelet, 4)
                tol = 0
            else:
                want = O.forward(x.astype(np.float64), wavelet, 4)
                tol = FLOAT_TOL
            assert_bands(gpu_bands(coeffs[k]), want, tol, (wavelet, k, sizes[k]))
        plan.close()
        del imgs, coeffs, plan
        torch.cuda.empty_cache()
