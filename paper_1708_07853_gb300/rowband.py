"""Row-band split of one image over several ranks: the forward transform with each rank
holding a band of rows, one halo exchange per level.

The paper's scheme is stated for any tiling of the image (Sec. 3, Sec. 5): each spatial step
reads a fixed neighbourhood, so a band of rows can be transformed on its own once it holds the
rows its outputs read.  Here each rank owns a band of image rows aligned to 2^J, so the band
boundaries stay on quad rows at every level.  At level j:

* a rank holds its rows of LL_{j-1};
* it sends its first and last `halo` rows to the ranks above and below, and receives theirs;
* it transforms the extended band [its rows, with the received rows above and below] as a
  plane, with the usual whole-sample-symmetric boundary at the plane's edges;
* it keeps the output rows that belong to its own band.

The halo is 2 kLag pixel rows: kLag lifting pairs (1 for CDF 5/3, 2 for CDF 9/7), each
reaching one quad row up and down.  Outputs that the artificial edge of an extended band
affects lie exactly kLag quad rows from that edge.  Those are the neighbour's rows, which it
computes itself.  At the image's own top and bottom edges nothing is received, and the plane's
symmetric boundary is the image's.

The arithmetic of a level is a callable, `level_fn(plane) -> (LL, HL, LH, HH)`.  On GPUs it is
the library's one-level forward (`dwt2_level`); the CPU tests pass the oracle.  The exchange
uses torch.distributed point-to-point messages.  Those run on gloo for CPU tensors and on NCCL
for CUDA tensors (one process per GPU).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def halo_rows(wavelet) -> int:
    """Pixel rows a level reads beyond the rows it outputs, on each side."""
    w = wavelet if isinstance(wavelet, str) else {0: "cdf53_int", 1: "cdf53", 2: "cdf97"}[int(wavelet)]
    return 4 if w == "cdf97" else 2


def band_rows(H: int, levels: int, world: int, rank: int):
    """Rows [r0, r1) of an H-row image owned by `rank` of `world`: whole units of 2^levels rows,
    spread as evenly as possible (the last band takes the remainder)."""
    unit = 1 << levels
    units = (H + unit - 1) // unit
    base, extra = divmod(units, world)
    start = rank * base + min(rank, extra)
    stop = (rank + 1) * base + min(rank + 1, extra)
    return min(H, unit * start), min(H, unit * stop)


def check_bands(H: int, levels: int, world: int, wavelet) -> None:
    """The halo of every level must come from the adjacent band alone: each band holds at least
    `halo` rows of every level's input plane (raises ValueError otherwise)."""
    halo = halo_rows(wavelet)
    for rank in range(world):
        r0, r1 = band_rows(H, levels, world, rank)
        for j in range(1, levels + 1):
            a, b = r0 >> (j - 1), -(-r1 >> (j - 1))
            if world > 1 and b - a < halo:
                raise ValueError(
                    f"band {rank} has {b - a} rows at level {j}; the halo needs {halo}: "
                    f"use fewer ranks or fewer levels for {H} rows")


def _exchange(cur: torch.Tensor, halo: int, rank: int, world: int, group=None):
    """(rows received from the rank above, rows received from the rank below); empty at the
    image's edges."""
    empty = cur[:0]
    top = bottom = empty
    reqs = []
    if rank > 0:
        top = torch.empty_like(cur[:halo])
        reqs.append(dist.isend(cur[:halo].contiguous(), rank - 1, group=group))
        reqs.append(dist.irecv(top, rank - 1, group=group))
    if rank < world - 1:
        bottom = torch.empty_like(cur[-halo:])
        reqs.append(dist.isend(cur[-halo:].contiguous(), rank + 1, group=group))
        reqs.append(dist.irecv(bottom, rank + 1, group=group))
    for r in reqs:
        r.wait()
    return top, bottom


def forward_rowband(band: torch.Tensor, H: int, wavelet, levels: int, level_fn, rank: int,
                    world: int, group=None):
    """This rank's share of the J-level forward transform of an H-row image.

    band: the rank's rows band_rows(H, levels, world, rank) of the image, as a 2-D tensor.
    Returns (LL_J rows, [(HL_j, LH_j, HH_j) rows for j = 1..J]): the rows of every band that
    fall in this rank's band, in the layout of the whole image's bands (LL / HL rows
    [a/2, ceil(b/2)), LH / HH rows [a/2, floor(b/2)) for the band's rows [a, b) of a level's
    input)."""
    check_bands(H, levels, world, wavelet)
    halo = halo_rows(wavelet)
    r0, r1 = band_rows(H, levels, world, rank)
    if band.shape[0] != r1 - r0:
        raise ValueError(f"rank {rank} owns rows [{r0}, {r1}); got {band.shape[0]} rows")
    cur = band
    h = H
    details = []
    for j in range(1, levels + 1):
        a, b = r0 >> (j - 1), min(h, -(-r1 >> (j - 1)))
        top, bottom = _exchange(cur, halo, rank, world, group) if world > 1 else (cur[:0], cur[:0])
        ext = torch.cat([top, cur, bottom], dim=0)
        LL, HL, LH, HH = level_fn(ext)
        off = top.shape[0] // 2  # ext's quad row 0 is the image's quad row (a - top rows) / 2
        ne = -(-b // 2) - a // 2  # even rows (LL, HL) of this band
        no = b // 2 - a // 2      # odd rows (LH, HH)
        details.append((HL[off:off + ne], LH[off:off + no], HH[off:off + no]))
        cur = LL[off:off + ne]
        h = (h + 1) // 2
    return cur, details


def dwt2_level(wavelet, band_dtype=None):
    """level_fn for CUDA tensors: one level of the library's forward (fp32 or int32 planes)."""
    from . import dwt2 as D

    def level(plane: torch.Tensor):
        c = D.forward(plane.contiguous(), wavelet, 1, band_dtype=band_dtype)
        return tuple(v.clone() for v in c.band_views())

    return level
