"""r-NN queries of new points from the stored grids (Sec. V) through the C ABI, against the
CPU oracle's oracle_rtg_query: the answer CSR must be identical, row by row."""
import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = rtg.Context(0)
    yield c
    c.close()


def _queries(seed, pts, k_new, d, dtype=np.float64):
    """New points in and around the unit cube, copies of indexed points, points a hair away
    from indexed points, and points far outside every grid's occupied cells."""
    rng = np.random.default_rng(seed)
    inside = rng.random((k_new, d))
    around = rng.uniform(-0.3, 1.3, (k_new // 2, d))
    copies = pts[rng.integers(0, len(pts), 40)].astype(np.float64)
    nudged = copies + rng.normal(0.0, 1e-7, copies.shape)
    far = rng.random((5, d)) + 50.0
    q = np.concatenate([inside, around, copies, nudged, far]).astype(dtype)
    return q


def _compare(res, ref):
    rp, col = res.download()
    assert np.array_equal(rp, ref.row_ptr), "row pointers differ"
    assert np.array_equal(col, ref.col), "answers differ"


@pytest.mark.parametrize("n,d,m,dtype", [(20000, 6, 8, np.float64), (5000, 3, 5, np.float32),
                                         (3000, 3, 64, np.float64), (2500, 12, 4, np.float64)])
def test_queries_match_oracle(ctx, n, d, m, dtype):
    pts = gen.points_uniform(50 + d, n, d, dtype)
    r = gen.radius_for_degree(n, d)
    T = gen.transforms(60 + m, d, m, r)
    ix = ctx.index(pts, r, T, r)
    q = _queries(70 + d, pts, 400, d, dtype)
    res = ix.query(q)
    ref = oracle.rtg_query(pts, r, T, r, q)
    _compare(res, ref)
    assert ref.nnz > 0
    # a copy of an indexed point finds at least itself; far points find nothing
    rows = res.download()[0]
    assert np.all(np.diff(rows)[-5:] == 0)
    res.release()
    ix.close()


def test_queries_on_device_and_points_as_queries(ctx):
    import torch
    n, d, m = 8000, 6, 8
    pts = gen.points_uniform(81, n, d)
    r = gen.radius_for_degree(n, d)
    T = gen.transforms(82, d, m, r)
    ix = ctx.index(torch.from_numpy(pts).cuda(), r, T, r)
    res = ix.query(torch.from_numpy(pts[:3000]).cuda())
    _compare(res, oracle.rtg_query(pts, r, T, r, pts[:3000]))
    # querying the points themselves: each point plus its neighbours in the RTG pair set
    rp, col = res.download()
    full = ctx.all_pairs(pts, r, T, r, symmetric=True)
    frp, fcol = full.download()
    for i in range(0, 3000, 97):
        want = np.sort(np.append(fcol[frp[i]:frp[i + 1]], i))
        assert np.array_equal(col[rp[i]:rp[i + 1]], want)
    full.release()
    res.release()
    ix.close()


def test_shift_only_grids_and_wider_cells(ctx):
    n, d, m = 6000, 6, 20
    pts = gen.points_uniform(91, n, d)
    r = gen.radius_for_degree(n, d)
    c = 1.35 * r
    T = gen.transforms(92, d, m, c, gen.SHIFT_ONLY)
    ix = ctx.index(pts, r, T, c)
    q = _queries(93, pts, 300, d)
    _compare(ix.query(q), oracle.rtg_query(pts, r, T, c, q))
    ix.close()


def test_dense_cells_take_warp_queries(ctx):
    # a tight cluster: cells of hundreds of points, so the index answers with a warp per query
    rng = np.random.default_rng(97)
    d, m, n = 3, 4, 6000
    pts = np.clip(rng.normal(0.5, 0.02, (n, d)), 0.0, 1.0)
    r = 0.03
    T = gen.transforms(98, d, m, r)
    ix = ctx.index(pts, r, T, r)
    q = np.concatenate([np.clip(rng.normal(0.5, 0.03, (300, d)), 0.0, 1.0), pts[:30]])
    res = ix.query(q)
    ref = oracle.rtg_query(pts, r, T, r, q)
    _compare(res, ref)
    assert ref.nnz > 300 * 50  # dense answers
    res.release()
    ix.close()


def test_empty_cases_and_errors(ctx):
    d, m = 3, 4
    pts = gen.points_uniform(95, 1000, d)
    r = gen.radius_for_degree(1000, d)
    T = gen.transforms(96, d, m, r)
    ix = ctx.index(pts, r, T, r)
    empty = ix.query(np.zeros((0, d)))
    assert empty.n == 0 and empty.nnz == 0
    empty.release()
    bad = np.full((3, d), 0.5)
    bad[1, 2] = np.nan
    with pytest.raises(rtg.RTGError):
        ix.query(bad)
    # the context stays usable after the refused query
    res = ix.query(pts[:10])
    assert res.nnz >= 10
    res.release()
    ix.close()
    ix0 = ctx.index(np.zeros((0, d)), r, T, r)
    res = ix0.query(pts[:5])
    rp, col = res.download()
    assert res.nnz == 0 and np.array_equal(rp, np.zeros(6, dtype=np.int64))
    res.release()
    ix0.close()
