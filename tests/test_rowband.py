"""The row-band split (paper_1708_07853_gb300/rowband.py) on CPU with gloo ranks: each rank
transforms its band of rows with one halo exchange per level, and the pieces put together are
the whole image's transform.  The level arithmetic is the oracle's one-level forward; each
owned output reads the same values as in the whole image, so the comparison is bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1708_07853_gb300 import rowband as RB


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _image(H, W, wavelet, seed):
    rng = np.random.default_rng(seed)
    if wavelet == "cdf53_int":
        return rng.integers(-(2 ** 15), 2 ** 15, (H, W)).astype(np.int64)
    return rng.uniform(0, 255, (H, W))


def _rank(rank, world, port, cases, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O

    out = []
    for H, W, wavelet, levels, seed in cases:
        x = _image(H, W, wavelet, seed)
        r0, r1 = RB.band_rows(H, levels, world, rank)

        def level_fn(plane):
            return tuple(torch.from_numpy(np.ascontiguousarray(b))
                         for b in O.forward(plane.numpy(), wavelet, 1))

        ll, det = RB.forward_rowband(torch.from_numpy(x[r0:r1]), H, wavelet, levels, level_fn,
                                     rank, world)
        out.append((ll.numpy(), [tuple(t.numpy() for t in d) for d in det]))
    q.put((rank, out))
    dist.destroy_process_group()


CASES = [(200, 37, "cdf97", 3, 1), (200, 37, "cdf53_int", 3, 2), (257, 64, "cdf53", 4, 3),
         (131, 19, "cdf97", 2, 4), (96, 9, "cdf53_int", 4, 5)]


@pytest.mark.parametrize("world", [2, 3])
def test_rowband_forward_equals_whole_image(world):
    from oracle import oracle as O

    cases = [c for c in CASES if _fits(c, world)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k, (H, W, wavelet, levels, seed) in enumerate(cases):
        want = O.forward(_image(H, W, wavelet, seed), wavelet, levels)
        ll = np.concatenate([res[r][k][0] for r in range(world)], axis=0)
        assert np.array_equal(ll, want[0]), (H, W, wavelet, levels)
        for j in range(1, levels + 1):
            got = [np.concatenate([res[r][k][1][j - 1][b] for r in range(world)], axis=0)
                   for b in range(3)]
            base = 1 + 3 * (levels - j)
            for b in range(3):
                assert np.array_equal(got[b], want[base + b]), (H, W, wavelet, levels, j, b)


def _fits(case, world):
    H, _, wavelet, levels, _ = case
    try:
        RB.check_bands(H, levels, world, wavelet)
        return True
    except ValueError:
        return False


def test_band_rows_partition_and_alignment():
    for H, J, world in [(200, 3, 2), (8192, 5, 8), (1000, 4, 3), (64, 2, 5)]:
        rows = [RB.band_rows(H, J, world, r) for r in range(world)]
        assert rows[0][0] == 0 and rows[-1][1] == H
        for (a0, a1), (b0, b1) in zip(rows, rows[1:]):
            assert a1 == b0
        for r0, r1 in rows[:-1]:
            assert r0 % (1 << J) == 0 and r1 % (1 << J) == 0
    assert RB.halo_rows("cdf97") == 4 and RB.halo_rows("cdf53_int") == 2


def test_thin_bands_are_rejected():
    # 64 rows over 5 ranks at 3 levels: bands of 8 or 16 rows, 1-2 rows at level 3 < halo 4
    with pytest.raises(ValueError):
        RB.check_bands(64, 3, 5, "cdf97")
    RB.check_bands(8192, 5, 8, "cdf97")  # the 8-GPU split of the 8192^2 image is fine
