"""Host logic of the window kernel's launch plan (no GPU): the tile schedule
from bz_tile_schedule covers every row of every 256-column tile column exactly
once, stays within one wave of resident warps, and gives the two edge columns
shorter tiles only where the balanced schedule applies."""
import ctypes

import numpy as np
import pytest

COLS = 256


@pytest.fixture(scope="module")
def lib():
    import paper_1905_13038_gb300 as bz
    L = ctypes.CDLL(bz.build())
    L.bz_tile_schedule.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    L.bz_tile_schedule.restype = ctypes.c_int32
    return L


def plan(L, H, W, sms, pipe, stripes):
    out = (ctypes.c_int64 * 6)()
    assert L.bz_tile_schedule(H, W, sms, pipe, stripes, out) == 0
    return dict(zip(["tiles_x", "tile_h", "edge_h", "n_edge", "total", "resident"], list(out)))


def tiles(p, H):
    """Decode every tile index: edge tiles first (left and right column in
    turn, edge_h rows each), then the interior columns in tile_h rows."""
    tx_n, th, eh, ne, total = p["tiles_x"], p["tile_h"], p["edge_h"], p["n_edge"], p["total"]
    for t in range(total):
        if t < ne:
            tx = tx_n - 1 if t & 1 else 0
            y0 = (t >> 1) * eh
            y1 = y0 + eh
        else:
            t2 = t - ne
            ncol = tx_n - 2 if ne else tx_n
            ty, r = divmod(t2, ncol)
            tx = (1 if ne else 0) + r
            y0 = ty * th
            y1 = y0 + th
        yield tx, y0, min(y1, H)


CASES = [
    # H, W, SMs
    (3072, 4096, 152),
    (3366, 4760, 152),
    (4096, 3072, 152),
    (384, 512, 152),
    (20000, 8, 152),
    (3000, 1000, 152),
    (5000, 260, 152),
    (1, 700, 152),
    (700, 1, 152),
    (12000, 40000, 152),
    (3072, 4096, 132),
    (777, 2049, 16),
]


@pytest.mark.parametrize("H,W,sms", CASES)
@pytest.mark.parametrize("pipe", [0, 1])
@pytest.mark.parametrize("stripes", [0, 1])
def test_schedule_covers_every_row_once(lib, H, W, sms, pipe, stripes):
    p = plan(lib, H, W, sms, pipe, stripes)
    assert p["tiles_x"] == (W + COLS - 1) // COLS
    assert p["resident"] == sms * 16
    cover = np.zeros((p["tiles_x"], H), np.int32)
    for tx, y0, y1 in tiles(p, H):
        assert 0 <= tx < p["tiles_x"] and 0 <= y0 < y1 <= H
        cover[tx, y0:y1] += 1
    assert (cover == 1).all()
    uniform = p["tiles_x"] * -(-H // p["tile_h"]) if not p["n_edge"] else None
    if p["n_edge"]:
        # balanced: only without stripes, with interior columns, shorter edges,
        # and still one wave
        assert not stripes and p["tiles_x"] >= 3
        assert p["edge_h"] < p["tile_h"]
        assert p["total"] <= p["resident"]
    else:
        assert p["edge_h"] == p["tile_h"] and p["total"] == uniform


def test_schedule_of_the_benchmark_page(lib):
    # 4096 x 3072 on 152 SMs, edge fraction 0.7 on the pipelined kernel: with
    # 21-row interior tiles (the shortest one-wave height) and 15-row edge
    # tiles (0.7 x 21 rounded) the grid would take 14 x 147 + 2 x 205 = 2468
    # warps, more than the 2432 resident; 22-row interior tiles with 15-row
    # edges take 14 x 140 + 2 x 205 = 2370
    p = plan(lib, 3072, 4096, 152, 1, 0)
    assert (p["tiles_x"], p["tile_h"], p["edge_h"], p["total"], p["resident"]) == (16, 22, 15, 2370, 2432)
    # the stripe launch keeps uniform 21-row tiles: 16 x 147
    p = plan(lib, 3072, 4096, 152, 1, 1)
    assert (p["tile_h"], p["n_edge"], p["total"]) == (21, 0, 2352)


def test_schedule_rejects_bad_arguments(lib):
    out = (ctypes.c_int64 * 6)()
    assert lib.bz_tile_schedule(0, 10, 152, 1, 0, out) == -1
    assert lib.bz_tile_schedule(10, 10, 0, 1, 0, out) == -1
    assert lib.bz_tile_schedule(10, 10, 152, 1, 0, None) == -1
