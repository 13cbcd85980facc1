"""The tile plan of the temporally tiled kernels, checked on the CPU.

A tiled launch advances every tile T steps with the light-cone halo
recomputed: tile b owns cells [b own, (b + 1) own), own = cells - 2T, and
holds the tile positions 0 .. cells - 1 starting at cell tb = b own - T.  The
tile that holds the last cell starts 4 or 8 cells earlier when that cell
would be its first owned cell or the first cell of a warp, because a
first-order Mur end reads its neighbour's new field, one cell beyond the
stencil's reach.  For every plan that `mbs_tile_plan` accepts, the model
below (the placement rule restated) must give:

* every cell of [0, nx) owned by exactly one tile, and written back once;
* every access of every tile inside the padded rows (PAD = 512 cells on
  each side, rows of ceil((nx + 2 PAD) / 32) * 32);
* the last cell's neighbour in the same warp and valid for all T steps
  (position >= T), and cell 0's neighbour likewise (position <= cells-1-T).

These are the conditions under which the kernels never read or write past
their rows and the absorbing ends read valid neighbours (Sec. 2.2, the Mur
condition of the boundary update).
"""
import math

import numpy as np
import pytest

import paper_2005_05412_gb300 as mbs
from paper_2005_05412_gb300 import build as mbs_build

PAD = 512


@pytest.fixture(scope="module", autouse=True)
def built():
    mbs_build.build()


def placement(nx, cells, T, span):
    """(tb, c_own) of every tile; of long grids only the first and last three
    (the tiles between start at b own - T and own a full tile, so the
    conditions below hold for them whenever they hold for their neighbours)."""
    own = cells - 2 * T
    n = math.ceil(nx / own)
    out = []
    for b in (range(n) if n <= 64 else list(range(3)) + list(range(n - 3, n))):
        c_own = b * own
        tb = c_own - T
        if nx - 1 < c_own + own:
            if nx - 1 == c_own or (nx - 1 - tb) % span == 0:
                tb -= 4
            if (nx - 1 - tb) % span == 0:
                tb -= 4
        out.append((tb, c_own))
    return out


def check_plan(n_levels, nx, cells, T, span):
    own = cells - 2 * T
    ld = (nx + 2 * PAD + 31) // 32 * 32
    tiles = placement(nx, cells, T, span)
    assert mbs.mbs_tile_plan(n_levels, cells, nx, T) == math.ceil(nx / own)
    covered = 0
    for tb, c_own in tiles:
        if c_own > covered:          # the regular tiles skipped on long grids
            assert c_own % own == 0
            covered = c_own
        lo = c_own - tb                                  # tile position of the first owned cell
        assert lo >= T, (nx, T, tb)
        # owned positions [lo, min(lo + own, cells - T)), written back below nx
        end = min(c_own + own, tb + cells - T, nx)
        assert c_own == covered, (nx, T, "gap or overlap")
        assert end == min(c_own + own, nx), (nx, T, "owned cells cut off by the light cone")
        covered = end
        assert tb >= -PAD and tb + cells <= ld - PAD, (nx, T, "access outside the padded rows")
    assert covered == nx
    tb_last = tiles[-1][0]
    p = nx - 1 - tb_last                                 # position of the last cell
    assert p >= T + 1 and p % span != 0, (nx, T, "last cell's neighbour")
    q = -tiles[0][0]                                     # position of cell 0
    assert q % span != span - 1 and q + 1 <= cells - 1 - T, (nx, T, "cell 0's neighbour")


def grids():
    rng = np.random.default_rng(7)
    return list(range(8, 1400)) + [int(x) for x in rng.integers(1400, 3_000_000, 40)] + [1_048_576, 262_144, 131_072]


@pytest.mark.parametrize("n_levels,span", [(2, 128), (3, 64)])
def test_cuda_core_tiles_every_grid(n_levels, span):
    """N = 2 (4 cells per lane, 512-cell tiles) and N = 3 (2 cells per lane):
    every multiple of 4 up to the documented maximum fits every grid."""
    t_max = 116 if n_levels == 2 else 52
    for nx in grids():
        for T in range(4, t_max + 1, 4):
            check_plan(n_levels, nx, 512, T, span)
    for bad in (0, 2, 6, t_max + 4):
        with pytest.raises(mbs.MBSError):
            mbs.mbs_tile_plan(n_levels, 512, 4096, bad)
    with pytest.raises(mbs.MBSError):
        mbs.mbs_tile_plan(n_levels, 256, 4096, 8)


@pytest.mark.parametrize("cells", [128, 256])
def test_tensor_core_tiles_accepted_plans_are_safe(cells):
    """N >= 4 (one cell per thread, warps of 32 cells): whatever the library
    accepts satisfies every condition; T = 1..20 (128-cell tiles) and 1..26
    (256-cell tiles) are accepted on every grid of at least 8 cells, as the
    header states."""
    always = 20 if cells == 128 else 26
    accepted = 0
    for nx in grids():
        for T in range(1, (cells - 32) // 2 + 1):
            try:
                mbs.mbs_tile_plan(6, cells, nx, T)
            except mbs.MBSError:
                assert T > always, (nx, T)
                continue
            accepted += 1
            check_plan(6, nx, cells, T, 32)
    assert accepted > 0.5 * len(grids()) * ((cells - 32) // 2)


def test_plan_rejects_bad_arguments():
    for args in [(1, 512, 4096, 8), (7, 128, 4096, 8), (6, 64, 4096, 8), (6, 128, 4, 8), (2, 512, 4, 8)]:
        with pytest.raises(mbs.MBSError) as e:
            mbs.mbs_tile_plan(*args)
        assert e.value.status == mbs.MBS_E_INVALID
