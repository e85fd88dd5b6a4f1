"""Bit-matrix dedupe (the flattened bit array of Sec. III-B): the union of every grid's
reported candidates through one bit per pair gives the same CSR as the first-grid rule and
the oracle's unordered sets, single and batched, upper and symmetric; larger instances are
refused."""
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


@pytest.mark.parametrize("n,d,m,dtype", [(2000, 3, 5, np.float64), (9001, 6, 8, np.float32),
                                         (16384, 2, 20, np.float64)])
def test_bitset_equals_oracle(ctx, n, d, m, dtype):
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(51 + d, n, d, dtype)
    T = gen.transforms(51 + d, d, m, r)
    res = ctx.all_pairs(pts, r, T, r, bitset=True)
    rp, col = res.download()
    st = res.stats
    res.release()
    ref = oracle.rtg(pts, r, T, r)
    assert np.array_equal(rp, ref.csr.row_ptr) and np.array_equal(col, ref.csr.col)
    assert st["pairs"] == ref.csr.nnz
    assert st["candidates"] == [s["candidates"] for s in ref.stats]


def test_bitset_symmetric_and_clustered(ctx):
    n, d, m = 5000, 3, 6
    pts = gen.points_mixture(53, n, d, k=3, sigma=0.02, dtype=np.float64)
    r = 0.04
    T = gen.transforms(53, d, m, r)
    a = ctx.all_pairs(pts, r, T, r, symmetric=True, bitset=True)
    b = ctx.all_pairs(pts, r, T, r, symmetric=True)
    ra, ca = a.download()
    rb, cb = b.download()
    assert a.stats["large_cells"] > 0
    assert np.array_equal(ra, rb) and np.array_equal(ca, cb)
    a.release()
    b.release()


def test_bitset_batch_matches_single_builds(ctx):
    items = []
    for i, (n, d) in enumerate([(1500, 3), (4000, 6), (700, 9), (12000, 2)]):
        r = gen.radius_for_degree(n, d)
        items.append((gen.points_uniform(60 + i, n, d, np.float32), r,
                      gen.transforms(60 + i, d, 6, r), r))
    res, offs = ctx.batch_all_pairs(items, m=6, bitset=True)
    rp, col = res.download()
    res.release()
    for b, (p, r, T, c) in enumerate(items):
        ref = oracle.rtg(p, r, T, c).csr
        lo, hi = offs[b], offs[b + 1]
        got_rp = rp[lo:hi + 1] - rp[lo]
        got_col = col[rp[lo]:rp[hi]] - lo
        assert np.array_equal(got_rp, ref.row_ptr) and np.array_equal(got_col, ref.col)


def test_bitset_refuses_large_instances(ctx):
    pts = gen.points_uniform(70, 16385, 2)
    T = gen.transforms(70, 2, 2, 0.01)
    with pytest.raises(rtg.RTGError):
        ctx.all_pairs(pts, 0.01, T, 0.01, bitset=True)
