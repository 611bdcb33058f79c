"""The claim order of the fused ME + checks launch (no GPU: rfsr_fused_schedule is host code).

The launch's CTAs claim tiles in this order, and a check tile waits for the ME bands it reads.
No CTA can then wait forever only if every ME tile that a check tile depends on comes earlier in
the order (the lowest unfinished tile can always proceed).  The dependencies are derived here
from the tile geometry the header states, independently of the library: a 32 x 32 check tile at
tile row r reads the motion fields of rows 32 r - 2 .. 32 r + 33 (the 3 x 3 median's halo of its
32 rows plus one), which lie in the 64-row ME bands of those rows, every 120-column tile and
every past frame of each."""
import itertools

import numpy as np
import pytest

from paper_2203_09200_gb300 import rfsr


def decode(items):
    cc = (items >> 31) & 1
    col = items & 0x3FF
    row = (items >> 10) & 0xFFF
    k = (items >> 22) & 3
    return cc.astype(bool), col.astype(int), row.astype(int), k.astype(int)


@pytest.mark.parametrize("H,W,K,grid", [(1080, 1920, 3, 304), (720, 1280, 2, 304), (64, 64, 1, 304),
                                        (130, 246, 3, 16), (16, 16, 1, 1), (2160, 3840, 3, 608),
                                        (8192, 200, 2, 304)])
def test_every_tile_once_and_dependencies_first(H, W, K, grid):
    try:
        items = rfsr.fused_schedule(H, W, K, grid)
    except RuntimeError as e:            # the library is not built in this checkout
        pytest.skip(str(e))
    cc, col, row, k = decode(items)
    nb, nc = -(-H // 64), -(-W // 120)
    ny, nx = -(-H // 32), -(-W // 32)
    me = sorted(zip(row[~cc], col[~cc], k[~cc]))
    assert me == sorted(itertools.product(range(nb), range(nc), range(K))), "ME tiles"
    checks = sorted(zip(row[cc], col[cc]))
    assert checks == sorted(itertools.product(range(ny), range(nx))), "check tiles"
    # position of the last ME tile of each band
    last = np.full(nb, -1)
    for i in np.nonzero(~cc)[0]:
        last[row[i]] = max(last[row[i]], i)
    for i in np.nonzero(cc)[0]:
        r = row[i]
        y_lo, y_hi = max(0, 32 * r - 2), min(H - 1, 32 * r + 33)
        for b in range(y_lo // 64, y_hi // 64 + 1):
            assert last[b] < i, f"check tile row {r} at {i} before ME band {b} (last at {last[b]})"


def test_bad_arguments():
    try:
        rfsr.load()
    except RuntimeError as e:
        pytest.skip(str(e))
    with pytest.raises(rfsr.RfsrError, match="EINVAL"):
        rfsr.fused_schedule(8, 64, 1, 304)
    with pytest.raises(rfsr.RfsrError, match="EINVAL"):
        rfsr.fused_schedule(64, 64, 0, 304)
