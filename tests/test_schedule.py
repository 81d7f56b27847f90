"""Host logic of the persistent step kernel's tile schedule
(``lbm_plan_tiles``): every tile of every lattice is dealt exactly once,
each block walks runs of tiles down one tile column, tall columns are cut
so that one large lattice still reaches every block, and the load stays
balanced.  No GPU needed."""
import math

import numpy as np
import pytest

from paper_1309_6726_gb300 import inputs as I
from paper_1309_6726_gb300 import lbm


def _runs(sched, grid, ty):
    """Per block: its tiles in order and its maximal runs of consecutive
    tiles down one tile column."""
    blocks = []
    for b in range(grid):
        col = sched[:, b, :]
        n = int(np.argmax(col[:, 0] < 0)) if (col[:, 0] < 0).any() else len(col)
        # nothing after a block's end marker
        assert (col[n:, 0] == -1).all()
        tiles = [tuple(int(v) for v in t) for t in col[:n]]
        runs = []
        for t in tiles:
            if runs and runs[-1][-1][0] == t[0] and runs[-1][-1][1] == t[1] \
                    and t[2] == runs[-1][-1][2] + ty:
                runs[-1].append(t)
            else:
                runs.append([t])
        blocks.append((tiles, runs))
    return blocks


def _check(sizes, tx, ty, grid):
    sched = lbm.plan_tiles(sizes, tx, ty, grid)
    assert sched.shape[1:] == (grid, 3)
    blocks = _runs(sched, grid, ty)
    dealt = [t for tiles, _ in blocks for t in tiles]
    expect = [(l, cx * tx, ry * ty)
              for l, (nx, ny) in enumerate(sizes)
              for cx in range(math.ceil(nx / tx))
              for ry in range(math.ceil(ny / ty))]
    # every tile exactly once
    assert len(dealt) == len(expect)
    assert sorted(dealt) == sorted(expect)
    total = len(expect)
    seg = max(4, math.ceil(total / (4 * grid)))
    rows = [math.ceil(ny / ty) for _, ny in sizes]
    for tiles, runs in blocks:
        for run in runs:
            # whole strips: a run starts on a multiple of the strip length
            # and ends on one or at the column's end
            r0 = run[0][2] // ty
            r1 = r0 + len(run)
            assert r0 % seg == 0
            assert r1 % seg == 0 or r1 == rows[run[0][0]]
    loads = [len(tiles) for tiles, _ in blocks]
    # longest-first greedy: no block exceeds the mean by more than a strip
    assert max(loads) <= math.ceil(total / grid) + seg
    return sched, blocks, seg


def test_single_tall_lattice_reaches_every_block():
    # the 2048 x 2048 preform: 32 tile columns of 256 tiles at 64 x 8
    sched, blocks, seg = _check([(2048, 2048)], 64, 8, 152)
    assert seg == 14
    loads = [len(t) for t, _ in blocks]
    assert min(loads) > 0
    assert max(loads) - min(loads) <= seg
    # an uncut column schedule would leave 120 of 152 blocks idle
    assert sched.shape[0] < 256


def test_paper_scale_capillary_fp16_tiles():
    # 4096 x 128 at 64 x 4 over 304 blocks: columns of 32 tiles cut to 4
    _, blocks, seg = _check([(4096, 128)], 64, 4, 304)
    assert seg == 4
    assert all(len(run) == 4 for _, runs in blocks for run in runs)


def test_sweep_columns_stay_whole():
    # the 512-capillary sweep: short columns, never cut
    members = I.sweep_members(512)
    sizes = [(m.length + 64 + 32, m.width + 2) for m in members]
    for tx, ty, grid in ((64, 8, 152), (64, 4, 304)):
        sched, blocks, seg = _check(sizes, tx, ty, grid)
        rows = {l: math.ceil(ny / ty) for l, (_, ny) in enumerate(sizes)}
        assert seg > max(rows.values())
        for _, runs in blocks:
            for run in runs:
                assert len(run) == rows[run[0][0]]
        loads = [len(t) for t, _ in blocks]
        # many short strips balance closely
        assert max(loads) - min(loads) <= max(rows.values())


@pytest.mark.parametrize("sizes,tx,ty,grid", [
    ([(1, 3)], 32, 4, 8),                      # one node column, one tile
    ([(37, 23), (130, 11), (5, 400)], 32, 8, 3),  # ragged edges, few blocks
    ([(64, 8)] * 7, 64, 8, 16),                # more blocks than tiles
    ([(200, 900), (33, 2)], 128, 4, 5),
])
def test_ragged_and_degenerate_batches(sizes, tx, ty, grid):
    _check(sizes, tx, ty, grid)


def test_plan_tiles_rejects_bad_arguments():
    with pytest.raises(lbm.LbmError):
        lbm.plan_tiles([], 64, 8, 152)
    with pytest.raises(lbm.LbmError):
        lbm.plan_tiles([(64, 8)], 0, 8, 152)
    with pytest.raises(lbm.LbmError):
        lbm.plan_tiles([(64, 8)], 64, 8, 0)
    with pytest.raises(lbm.LbmError):
        lbm.plan_tiles([(0, 8)], 64, 8, 4)
    # an output buffer smaller than 3 * grid * slots values
    import ctypes as C
    lib = lbm.load_library()
    nx = (C.c_int32 * 1)(256)
    ny = (C.c_int32 * 1)(64)
    out = (C.c_int32 * 6)()
    slots = C.c_int32()
    assert lib.lbm_plan_tiles(nx, ny, 1, 64, 8, 2, out, 6,
                              C.byref(slots)) != lbm.LBM_OK
    assert slots.value == 16
