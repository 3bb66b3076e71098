"""Batched solver, host side (no GPU): the problem order and tile table of the
C library are bit-exact against the oracle's definition, the oracle's plan
keeps its invariants, and invalid batches are rejected before any device
work."""
import ctypes

import numpy as np
import pytest

from oracle import gsi_oracle as O
from paper_2306_10379_gb300 import inputs as I


def _gsi():
    from paper_2306_10379_gb300 import gsi
    try:
        gsi.lib()
    except Exception as e:  # pragma: no cover - the library is built by build()
        pytest.skip(f"libgsi.so not loadable: {e}")
    return gsi


@pytest.mark.parametrize("seed,tile_max,target", [(1, 128, 2432), (2, 512, 304), (3, 1000, 1216),
                                                  (4, 4096, 608), (5, 2048, 100000)])
def test_plan_matches_oracle(seed, tile_max, target):
    """The library's tile table equals the oracle's definition for every
    problem active and for a random active subset (where the finer tiles of
    a nearly finished batch appear)."""
    gsi = _gsi()
    n, p = I.batched_sizes(512, I.SEED_BASE + seed)
    act = (I.uniform53(512, I.SEED_BASE + seed, stream=9) < 0.05).astype(np.int32)
    for active in (None, act):
        order, tiles = gsi.batched_plan(n, p, tile_max, target, active)
        o_order, o_tiles = O.batched_plan(n, p, tile_max, target, active)
        assert order.tolist() == o_order
        assert tiles == o_tiles


def test_plan_ties_ragged_and_shrinking():
    gsi = _gsi()
    n = np.array([100, 300, 300, 64, 100, 257], np.int32)
    p = np.array([4, 32, 32, 2, 32, 8], np.int32)
    order, tiles = gsi.batched_plan(n, p, 64, 4)
    assert tiles == O.batched_plan(n, p, 64, 4)[1]
    # descending p, then descending n, ties by index
    assert order.tolist() == [1, 2, 4, 5, 0, 3]
    # S = 1121 rows over 4 target tiles -> T = 281; p = 32 -> 281-row tiles
    _, t = gsi.batched_plan(n, p, 4096, 4)
    assert t[:2] == [(1, 0, 281), (1, 281, 19)]
    # many target tiles: every problem at the 64-row floor
    _, t = gsi.batched_plan(n, p, 4096, 10 ** 6)
    assert [r for (i, _, r) in t if i == 5] == [64, 64, 64, 64, 1]
    assert [r for (i, _, r) in t if i == 1] == [64, 64, 64, 64, 44]


def test_oracle_plan_invariants():
    """Every row of every selected problem is in exactly one tile; a
    problem's tiles are adjacent and in row order; tile lengths respect
    tile_max and the 64-row floor."""
    n, p = I.batched_sizes(64, I.SEED_BASE + 9, 100, 5000)
    for tm, target in ((64, 10), (100, 500), (4096, 50), (4096, 10 ** 6)):
        order, tiles = O.batched_plan(n, p, tm, target)
        assert sorted(order) == list(range(n.size))
        seen = {}
        for prob, r0, rows in tiles:
            assert 1 <= rows <= tm
            seen.setdefault(prob, []).append((r0, rows))
        assert [t[0] for t in tiles] == [i for i in order for _ in range(len(seen[i]))]
        for i, segs in seen.items():
            cover = np.zeros(int(n[i]), int)
            for r0, rows in segs:
                cover[r0:r0 + rows] += 1
            assert np.all(cover == 1)
            assert [s[0] for s in segs] == sorted(s[0] for s in segs)
            full = [r for _, r in segs[:-1]]
            assert all(r >= min(tm, 64) for r in full)


def test_batch_sizes_distribution():
    n, p = I.batched_sizes(4096, I.SEED_BASE + 5)
    assert n.min() >= 2048 and n.max() <= 65536
    assert set(np.unique(p).tolist()) == {4, 8, 16, 32}
    assert abs(n.mean() - (2048 + 65536) / 2) < 0.03 * 65536


def _create(gsi, n, p, rowptr, colidx, val, X0):
    L = gsi.lib()
    arrs = [np.ascontiguousarray(n, np.int32), np.ascontiguousarray(p, np.int32),
            np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(colidx, np.int32),
            np.ascontiguousarray(val, np.float32), np.ascontiguousarray(X0, np.float64)]
    ctx = ctypes.c_void_p()
    st = L.gsi_batched_create(len(arrs[0]), *(a.ctypes.data for a in arrs), None, None, None,
                              ctypes.byref(ctx))
    return st


def test_create_rejects_invalid_batches():
    """Checked on the host before any device allocation: block widths outside
    {2, 4, 8, 16, 32}, n < 2p, decreasing rowptr, column indices outside the
    problem."""
    gsi = _gsi()
    A = I.fd_laplacian((8,))
    good = dict(rowptr=A.rowptr, colidx=A.colidx, val=A.val, X0=np.ones(8 * 2))
    assert _create(gsi, [8], [3], **{**good, "X0": np.ones(24)}) == gsi.GSI_ERR_ARG
    assert _create(gsi, [8], [8], **{**good, "X0": np.ones(64)}) == gsi.GSI_ERR_ARG
    bad = A.colidx.copy()
    bad[5] = 8
    assert _create(gsi, [8], [2], **{**good, "colidx": bad}) == gsi.GSI_ERR_ARG
    rp = A.rowptr.copy()
    rp[3] = rp[4] + 1
    assert _create(gsi, [8], [2], **{**good, "rowptr": rp}) == gsi.GSI_ERR_ARG
