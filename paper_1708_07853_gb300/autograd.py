"""torch.autograd Functions over the library's forward / inverse transforms.

Both are linear, so nothing is saved for backward but the shapes: the backward of the forward
transform W is its transpose W^T (dwt2_forward_adjoint), the backward of the inverse W^-1 is
W^-T (dwt2_inverse_adjoint); every level's gradient is computed by the hand-written adjoint
kernels, from the coarsest level down (W^T) or from the finest up (W^-T).

Coefficients travel as one flat float32 tensor per image, laid out exactly as dwt2_layout
describes (fp32 storage makes every band, and the padding between rows and bands, a whole
number of floats).  `band_views` gives the LL / HL / LH / HH planes as views into it; the
padding entries are zero in forward outputs and in gradients.  The kernels write the bands
only, so outputs are allocated uninitialised and just their padding entries are zeroed, from an
index cached per layout (empty when the widths are multiples of 4 and the band sizes multiples of
256 bytes, as for 1024 x 1024 images).  All images of a call go through the uniform-batch entry
points: one launch per level covers every image.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dwt2 as D


def coeff_floats(H: int, W: int, levels: int) -> int:
    _, nbytes = D.layout(H, W, levels, D.DT_F32)
    return nbytes // 4


_PAD = {}


def padding_index(H: int, W: int, levels: int, device) -> torch.Tensor:
    """Positions of the flat coefficient layout that belong to no band (row padding and the gaps
    that align each band to 256 bytes), as a cached int64 tensor on device."""
    key = (H, W, levels, str(device))
    if key not in _PAD:
        lay, nbytes = D.layout(H, W, levels, D.DT_F32)
        pad = np.ones(nbytes // 4, dtype=bool)
        for b in lay:
            if b.h and b.w:
                o, p = b.offset_bytes // 4, b.pitch_bytes // 4
                pad[(o + np.arange(b.h)[:, None] * p + np.arange(b.w)[None, :]).ravel()] = False
        _PAD[key] = torch.from_numpy(np.nonzero(pad)[0]).to(device)
    return _PAD[key]


def _new_coeffs(n_img: int, H: int, W: int, levels: int, device) -> torch.Tensor:
    """Uninitialised flat coefficients whose padding entries are zero (the kernels then write
    every band entry)."""
    out = torch.empty((n_img, coeff_floats(H, W, levels)), dtype=torch.float32, device=device)
    pad = padding_index(H, W, levels, device)
    if pad.numel():
        out[:, pad] = 0.0
    return out


def band_views(c: torch.Tensor, H: int, W: int, levels: int):
    """Band planes (LL_J, then HL_j, LH_j, HH_j for j = J..1) as views into a flat coefficient
    tensor of shape (..., coeff_floats)."""
    lay, _ = D.layout(H, W, levels, D.DT_F32)
    out = []
    for b in lay:
        o, p = b.offset_bytes // 4, b.pitch_bytes // 4
        if b.h == 0 or b.w == 0:
            out.append(c[..., :0].reshape(*c.shape[:-1], b.h, b.w))
            continue
        out.append(c[..., o:o + b.h * p].reshape(*c.shape[:-1], b.h, p)[..., :b.w])
    return out


def _images(t: torch.Tensor):
    return t.reshape(-1, t.shape[-2], t.shape[-1])


def _check(x: torch.Tensor):
    if not x.is_cuda or x.dtype != torch.float32:
        raise ValueError("DWT2Fn / IDWT2Fn need float32 CUDA tensors")


class DWT2Fn(torch.autograd.Function):
    """c = W x for every image of x (..., H, W); c has shape (..., coeff_floats)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, wavelet: str, levels: int):
        _check(x)
        H, W = x.shape[-2:]
        xs = _images(x.contiguous())
        n = coeff_floats(H, W, levels)
        out = _new_coeffs(xs.shape[0], H, W, levels, x.device)
        D.forward_batch(xs, wavelet, levels, D.DT_F32, out=out)
        ctx.meta = (H, W, wavelet, levels, x.shape)
        return out.reshape(*x.shape[:-2], n)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        H, W, wavelet, levels, xshape = ctx.meta
        gs = g.reshape(-1, g.shape[-1]).contiguous()
        gx = D.forward_adjoint_batch(gs, H, W, wavelet, levels)
        return gx.reshape(xshape), None, None


class IDWT2Fn(torch.autograd.Function):
    """x = W^-1 c for every coefficient row of c (..., coeff_floats); x has shape (..., H, W)."""

    @staticmethod
    def forward(ctx, c: torch.Tensor, H: int, W: int, wavelet: str, levels: int):
        _check(c)
        cs = c.reshape(-1, c.shape[-1]).contiguous()
        x = D.inverse_batch(cs, H, W, wavelet, levels, D.DT_F32, img_dtype=torch.float32)
        ctx.meta = (H, W, wavelet, levels, c.shape)
        return x.reshape(*c.shape[:-1], H, W)

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        H, W, wavelet, levels, cshape = ctx.meta
        gxs = _images(gx.contiguous())
        gc = _new_coeffs(gxs.shape[0], H, W, levels, gx.device)
        D.inverse_adjoint_batch(gxs, wavelet, levels, out=gc)
        return gc.reshape(cshape), None, None, None, None


def dwt2(x: torch.Tensor, wavelet: str = "cdf97", levels: int = 1) -> torch.Tensor:
    return DWT2Fn.apply(x, wavelet, levels)


def idwt2(c: torch.Tensor, H: int, W: int, wavelet: str = "cdf97", levels: int = 1) -> torch.Tensor:
    return IDWT2Fn.apply(c, H, W, wavelet, levels)
