"""Seeded synthetic inputs, shared by the tests, the benchmark and the oracle checks.

This module holds no wavelet arithmetic: it only draws images.  The paper evaluates on FP32
images and tiles of 1024^2 to 8192^2 (Sec. 4) without naming a dataset; a seeded random field
with a 1/f^2 power spectrum (the spectrum of natural images) stands in for image content.

Recipe (field): z ~ N(0, 1) of shape H x W from numpy's default_rng(seed); Z = rfft2(z) * 1/|f|
with the DC term set to 0 (amplitude 1/f, power 1/f^2); v = irfft2(Z), min-max scaled to
[lo, hi]; for integer content rounded half-to-even.

`field_device` follows the same recipe on the GPU (torch's generator and FFT, fp32) for
benchmark workloads too large to draw on the host in seconds; its values differ from `field`'s
for the same seed, so tests that compare against the oracle draw with `field`.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1708_0000


def seed_for(config: int, image: int = 0) -> int:
    return SEED_BASE + 100 * config + image


def field(H: int, W: int, seed: int, lo: float = 0.0, hi: float = 255.0,
          integer: bool = True, dtype=np.float32) -> np.ndarray:
    """H x W seeded 1/f^2 random field scaled to [lo, hi] (rounded to integers if asked)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((H, W), dtype=np.float64)
    Z = np.fft.rfft2(z)
    del z
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = np.inf
    Z /= f
    del f
    v = np.fft.irfft2(Z, s=(H, W))
    del Z
    vmin, vmax = v.min(), v.max()
    if vmax > vmin:
        v = (v - vmin) * ((hi - lo) / (vmax - vmin)) + lo
    else:
        v = np.full((H, W), lo)
    if integer:
        v = np.rint(v)
    return v.astype(dtype)


def field_device(H: int, W: int, seed: int, device, lo: float = 0.0, hi: float = 255.0,
                 integer: bool = True):
    """`field`'s recipe drawn on a CUDA device (fp32 result); for benchmark-sized batches."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    z = torch.randn((H, W), generator=g, device=device, dtype=torch.float32)
    Z = torch.fft.rfft2(z)
    fy = torch.fft.fftfreq(H, device=device)[:, None]
    fx = torch.fft.rfftfreq(W, device=device)[None, :]
    f = torch.sqrt(fx * fx + fy * fy)
    f[0, 0] = float("inf")
    v = torch.fft.irfft2(Z / f, s=(H, W))
    vmin, vmax = v.min(), v.max()
    if float(vmax) > float(vmin):
        v = (v - vmin) * ((hi - lo) / (vmax - vmin)) + lo
    else:
        v = torch.full((H, W), lo, device=device)
    if integer:
        v = torch.round(v)
    return v.contiguous()


def field_plus_noise(H: int, W: int, seed: int, dtype=np.float32) -> np.ndarray:
    """0.5 * field + 0.5 * U[0, 255): non-integer content that stays in [0, 255]."""
    rng = np.random.default_rng(seed + 50)
    f = field(H, W, seed, integer=False, dtype=np.float64)
    u = rng.uniform(0.0, 255.0, (H, W))
    return (0.5 * f + 0.5 * u).astype(dtype)


def batch_sizes(n: int, seed: int, lo: int = 63, hi: int = 4096):
    """n (H, W) pairs, each side drawn independently log-uniform on [lo, hi] and rounded."""
    rng = np.random.default_rng(seed)
    s = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), (n, 2)))).astype(int)
    return [(int(h), int(w)) for h, w in s]


def random_ints(H: int, W: int, seed: int, lo: int = -(2 ** 15), hi: int = 2 ** 15) -> np.ndarray:
    return np.random.default_rng(seed).integers(lo, hi + 1, (H, W)).astype(np.int32)
