"""Multiple r-NN queries (Sec. II): neighbour lists of a subset of the points read from the
stored symmetric pair set.  The oracle's upper-triangular CSR fixes every list: the
neighbours of q are the columns of row q and the rows whose columns hold q."""
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


def _neighbours(csr, n):
    nb = [[] for _ in range(n)]
    for i in range(n):
        for j in csr.col[csr.row_ptr[i]:csr.row_ptr[i + 1]]:
            nb[i].append(int(j))
            nb[int(j)].append(i)
    return [sorted(x) for x in nb]


@pytest.mark.parametrize("on_device", [False, True])
def test_queries_match_the_oracle(ctx, on_device):
    n, d, m = 6007, 4, 6
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(31, n, d)
    T = gen.transforms(31, d, m, r)
    ref = _neighbours(oracle.rtg(pts, r, T, r).csr, n)
    g = ctx.all_pairs(pts, r, T, r, symmetric=True)
    rng = np.random.default_rng(5)
    q = np.concatenate([[0, n - 1, 17, 17], rng.integers(0, n, 3000)]).astype(np.int32)
    if on_device:
        import torch
        q_arg = torch.from_numpy(q).cuda()
    else:
        q_arg = q
    res = ctx.query_neighbors(g, q_arg)
    rp, col = res.download()
    assert len(rp) == len(q) + 1
    for k, v in enumerate(q):
        assert col[rp[k]:rp[k + 1]].tolist() == ref[v], (k, v)
    res.release()
    g.release()


def test_query_edge_cases(ctx):
    n, d = 3000, 3
    pts = gen.points_uniform(32, n, d)
    r = 0.05
    T = gen.transforms(32, d, 3, r)
    g = ctx.all_pairs(pts, r, T, r, symmetric=True)
    empty = ctx.query_neighbors(g, np.zeros(0, dtype=np.int32))
    rp, col = empty.download()
    assert rp.tolist() == [0] and len(col) == 0
    empty.release()
    with pytest.raises(rtg.RTGError):
        ctx.query_neighbors(g, np.array([0, n], dtype=np.int32))
    with pytest.raises(rtg.RTGError):
        ctx.query_neighbors(g, np.array([-1], dtype=np.int32))
    upper = ctx.all_pairs(pts, r, T, r)
    with pytest.raises(rtg.RTGError):
        ctx.query_neighbors(upper, np.array([0], dtype=np.int32))
    upper.release()
    # the context still works after the refused queries
    ok = ctx.query_neighbors(g, np.arange(n, dtype=np.int32))
    rp, col = ok.download()
    grp, gcol = g.download()
    assert np.array_equal(rp, grp) and np.array_equal(col, gcol)
    ok.release()
    g.release()
