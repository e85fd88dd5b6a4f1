"""The cell-major sort.  For one instance, where leaving the grid out of the sort key saves a
radix pass, the key kernel writes a grid-major copy of the cell indices, the sort orders
(cell, grid, point), and its last pass restores the composite keys and point indices.  The
reported pairs must be the oracle's bit for bit, and the same as the grid-major sort's
(RTG_CELL_MAJOR=0), in every output form; the index, which reads the sorted keys grid by grid,
must still get a grid-major sort."""
import os

import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu

_ENV = ("RTG_CELL_MAJOR", "RTG_SORT_VARIANT", "RTG_TUNE_CACHE", "RTG_AUTOTUNE")


def _context(cell_major: bool, variant: str | None = None):
    """A context created with the given switches (the environment is read at creation)."""
    old = {k: os.environ.get(k) for k in _ENV}
    try:
        for k in _ENV:
            os.environ.pop(k, None)
        if not cell_major:
            os.environ["RTG_CELL_MAJOR"] = "0"
        if variant:
            os.environ["RTG_SORT_VARIANT"] = variant
        return rtg.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def case100k():
    # the 100k workload of bench.py: 26-bit composite keys, 24-bit cell indices (3 passes, not 4)
    n, d, m = 100000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(0, n, d)
    T = gen.transforms(0, d, m, r)
    ref = oracle.rtg(pts, r, T, r)
    return pts, r, T, ref


def _build(ctx, pts, r, T, **kw):
    res = ctx.all_pairs(pts, r, T, r, **kw)
    rp, col = res.download()
    st = res.stats
    res.release()
    return rp, col, st


def _passes(bits, width=8):
    return -(-bits // width)


@pytest.mark.parametrize("variant", [None, "8,12,0", "8,16,1", "8,8,0", "8,12,2"],
                         ids=["tuned", "lookback-3072", "reduce-4096", "lookback-2048", "coop"])
def test_cell_major_sort_matches_the_oracle(case100k, variant):
    pts, r, T, ref = case100k
    ctx = _context(True, variant)
    try:
        # the first build, the second (the tuner's, unless a variant is forced) and a replay
        for _ in range(3):
            rp, col, st = _build(ctx, pts, r, T)
            assert np.array_equal(rp, ref.csr.row_ptr), "row pointers differ"
            assert np.array_equal(col, ref.csr.col), "columns differ"
            assert st["candidates"] == [s["candidates"] for s in ref.stats]
            assert st["max_cell"] == max(s["max_cell"] for s in ref.stats)
            sort = st["sort"]
            if variant == "8,12,2":
                # the single-launch sort keeps the grid in the key
                assert sort["cell_major"] == 0 and sort["sorted_bits"] == st["key_bits"]
            else:
                assert sort["cell_major"] == 1 and sort["digit_bits"] == 8
                assert sort["sorted_bits"] < st["key_bits"]
                assert st["sort_passes"] == _passes(sort["sorted_bits"]) < _passes(st["key_bits"])
    finally:
        ctx.close()


@pytest.mark.parametrize("kw", [dict(symmetric=True), dict(two_pass=True), dict(timing=True),
                                dict(on_device=True)], ids=["symmetric", "two_pass", "timing",
                                                            "on_device"])
def test_cell_major_equals_grid_major(case100k, kw):
    pts, r, T, _ = case100k
    kw = dict(kw)
    arg = pts
    if kw.pop("on_device", False):
        import torch
        arg = torch.from_numpy(pts).cuda()
    out = {}
    for cm in (True, False):
        ctx = _context(cm)
        try:
            for _ in range(2):  # the second build replays or tunes; both must agree
                rp, col, st = _build(ctx, arg, r, T, **kw)
                assert st["sort"]["cell_major"] == (1 if cm else 0)
                out.setdefault(cm, []).append((rp, col, st["candidates"], st["near_wall"]))
        finally:
            ctx.close()
    for (rp0, col0, c0, w0), (rp1, col1, c1, w1) in zip(out[True], out[False]):
        assert np.array_equal(rp0, rp1) and np.array_equal(col0, col1)
        assert c0 == c1 and w0 == w1


def test_index_after_a_cell_major_build_reads_grid_major_keys(case100k):
    # the index keeps the sort of its own build, which must be grid-major even on a context
    # whose builds of the same shape sorted cell-major
    pts, r, T, ref = case100k
    ctx = _context(True)
    try:
        rp, col, st = _build(ctx, pts, r, T)
        assert st["sort"]["cell_major"] == 1
        ix = ctx.index(pts, r, T, r)
        rng = np.random.default_rng(5)
        q = np.concatenate([rng.random((300, 6)), pts[rng.integers(0, len(pts), 50)]])
        res = ix.query(q)
        got_rp, got_col = res.download()
        res.release()
        want = oracle.rtg_query(pts, r, T, r, q)
        assert np.array_equal(got_rp, want.row_ptr) and np.array_equal(got_col, want.col)
        assert want.nnz > 0
        ix.close()
        # and a build after the index still sorts cell-major and matches the oracle
        rp, col, st = _build(ctx, pts, r, T)
        assert st["sort"]["cell_major"] == 1
        assert np.array_equal(rp, ref.csr.row_ptr) and np.array_equal(col, ref.csr.col)
    finally:
        ctx.close()
