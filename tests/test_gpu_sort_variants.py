"""Every compiled sort variant (digit width, tile size, pass strategy) and the autotuner that
chooses between them.  The sort is stable in every variant, so each must give the oracle's
CSR bit for bit; the autotuner must record its choice and reuse it from its JSON cache."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu

VARIANTS = [(bits, items, mode) for bits in (8, 9, 10, 11) for items in (8, 12, 16)
            for mode in (0, 1, 2)]
LOOKBACK_CODE = {0: 1, 1: 0, 2: 2}  # stats "lookback" of each pass strategy


def _context(env):
    """A context created with the given environment (read at creation)."""
    keys = ("RTG_SORT_VARIANT", "RTG_TUNE_CACHE", "RTG_AUTOTUNE", "RTG_TUNE_PAIRS_MAX_CAND")
    old = {k: os.environ.get(k) for k in keys}
    try:
        for k in keys:
            os.environ.pop(k, None)
        os.environ.update(env)
        return rtg.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def case32():
    # several hundred sort tiles and a ragged last tile: 37,003 points x 8 grids
    n, d, m = 37003, 4, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(21, n, d, np.float32)
    T = gen.transforms(21, d, m, r)
    ref = oracle.rtg(pts, r, T, r)
    return pts, r, T, ref


@pytest.fixture(scope="module")
def case64():
    # a composite key wider than 32 bits
    n, d, m = 6001, 6, 3
    pts = gen.points_uniform(22, n, d)
    r = 0.02
    T = gen.transforms(22, d, m, r)
    ref = oracle.rtg(pts, r, T, r)
    return pts, r, T, ref


def _check(ctx, pts, r, T, ref):
    res = ctx.all_pairs(pts, r, T, r)
    rp, col = res.download()
    st = res.stats
    res.release()
    assert np.array_equal(rp, ref.csr.row_ptr)
    assert np.array_equal(col, ref.csr.col)
    assert st["candidates"] == [s["candidates"] for s in ref.stats]
    return st


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: "bits%d-items%d-mode%d" % v)
def test_sort_variant_bit_exact(variant, case32, case64):
    ctx = _context({"RTG_SORT_VARIANT": "%d,%d,%d" % variant})
    try:
        st = _check(ctx, *case32)
        assert st["key_bits"] <= 32
        assert (st["sort"]["digit_bits"], st["sort"]["tile_keys"], st["sort"]["lookback"]) == \
            (variant[0], 256 * variant[1], LOOKBACK_CODE[variant[2]])
        # a cell-major sort (8-bit passes only) orders the cell index's bits alone
        assert st["sort_passes"] == -(-st["sort"]["sorted_bits"] // variant[0])
        if st["sort"]["cell_major"]:
            assert variant[0] == 8 and variant[2] != 2
            assert st["sort"]["sorted_bits"] < st["key_bits"]
        else:
            assert st["sort"]["sorted_bits"] == st["key_bits"]
        st = _check(ctx, *case64)
        assert st["key_bits"] > 32
        assert st["sort"]["digit_bits"] == variant[0]
    finally:
        ctx.close()


def test_autotuner_measures_once_and_caches(tmp_path, case32):
    path = str(tmp_path / "tune.json")
    ctx = _context({"RTG_TUNE_CACHE": path})
    try:
        st0 = _check(ctx, *case32)  # 296,024 keys: the first build takes the default
        assert st0["sort"]["tuned"] == 0 and st0["enumeration"]["tuned"] == 0
        st = _check(ctx, *case32)  # and the second measures every variant
        assert st["sort"]["tuned"] == 1 and st["attempts"] == 1
        assert st["enumeration"]["tuned"] == 1
        assert st["enumeration"]["spans_per_warp"] in (1, 2, 4)
        assert st["enumeration"]["dense_cell_min"] in (64, 128, 256)
        st2 = _check(ctx, *case32)
        assert st2["sort"] == st["sort"] and st2["enumeration"] == st["enumeration"]
    finally:
        ctx.close()
    doc = json.load(open(path))
    entries = doc["entries"]
    assert len(entries) == 1
    e = entries[0]
    assert e["elements"] == 37003 * 8 and e["key_bits"] == st["sort"]["sorted_bits"]
    assert (e["bits"], 256 * e["items"], LOOKBACK_CODE[e["mode"]]) == (
        st["sort"]["digit_bits"], st["sort"]["tile_keys"], st["sort"]["lookback"])
    assert e["us"] > 0
    # a new context takes the cached choice without measuring again
    ctx = _context({"RTG_TUNE_CACHE": path})
    try:
        st3 = _check(ctx, *case32)
        assert st3["sort"] == st["sort"]
    finally:
        ctx.close()
    assert json.load(open(path))["entries"] == entries


def test_autotune_off_takes_the_default(case32):
    ctx = _context({"RTG_AUTOTUNE": "0"})
    try:
        st = _check(ctx, *case32)
        assert st["sort"]["tuned"] == 0
        assert st["sort"]["digit_bits"] == 8 and st["sort"]["tile_keys"] == 2048
    finally:
        ctx.close()


@pytest.mark.parametrize("cap,tuned", [("1e6", 0), (None, 1)])
def test_enumeration_trials_are_capped_by_candidates(cap, tuned):
    # clustered points (cells of hundreds of points): above the candidate cap the second build
    # measures the sort variants only, since every enumeration trial would enumerate all the
    # candidates; under the default cap (4e9) this shape's enumeration is measured too
    n, d, m = 20000, 3, 8
    pts = gen.points_mixture(23, n, d, k=4, sigma=0.02, dtype=np.float32)
    r = gen.radius_for_degree(n, d)
    T = gen.transforms(23, d, m, r)
    ref = oracle.rtg(pts, r, T, r)
    ctx = _context({"RTG_TUNE_PAIRS_MAX_CAND": cap} if cap else {})
    try:
        st0 = _check(ctx, pts, r, T, ref)
        assert st0["total_candidates"] > 1e6
        st = _check(ctx, pts, r, T, ref)
        assert st["sort"]["tuned"] == 1
        assert st["enumeration"]["tuned"] == tuned
        st2 = _check(ctx, pts, r, T, ref)
        assert st2["enumeration"] == st["enumeration"]
    finally:
        ctx.close()
