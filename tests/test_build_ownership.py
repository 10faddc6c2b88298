"""The pyramid build's tile kernel stores every staged texel into the
hierarchy's copy of the map exactly once (CPU check of the ownership rule of
build_tiles: a 64 x 64-quad tile stages (tileQ + 1)^2 texels, owns its first
tileQ rows and columns, and the map's last row or column where that is the
tile's shared edge), for map sizes around the tile and pyramid boundaries and
each staging width (16-byte vectors of 2 FP32 or 4 FP16 texels, or single
texels when rows are not a multiple of the vector)."""

import numpy as np
import pytest


def top_level(n):
    L = 0
    while (1 << L) < n - 1:
        L += 1
    return max(L, 2)


def stores(n, vec):
    side = 1 << top_level(n)
    tq = min(side, 64)
    count = np.zeros((n, n), np.int64)
    for by in range(side // tq):
        for bx in range(side // tq):
            c0, r0 = bx * tq, by * tq
            for r in range(tq + 1):  # staged rows
                gr = r0 + r
                if gr >= n:
                    continue
                own_row = r < tq or gr == n - 1
                for v in range(tq // vec):  # vector loads of the first tq columns
                    gc = c0 + v * vec
                    if gc < n and own_row:
                        count[gr, gc:gc + vec] += 1
                gc = c0 + tq  # the shared last column
                if gc < n and gc == n - 1 and own_row:
                    count[gr, gc] += 1
    return count


@pytest.mark.parametrize("n", [2, 3, 5, 63, 64, 65, 66, 96, 100, 127, 128, 129, 130, 203, 256, 257, 300, 513])
def test_each_texel_stored_once(n):
    for vec in (1, 2, 4):
        if vec > 1 and n % vec:
            continue  # the kernel stages single texels then
        c = stores(n, vec)
        assert (c == 1).all(), (n, vec, np.argwhere(c != 1)[:5])
