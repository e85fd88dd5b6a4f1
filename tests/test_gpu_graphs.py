"""Replayed launch sequences (CUDA graphs): later builds of a shape replay the sequence
captured on an earlier one.  New points and transforms of the same shape, host or device
inputs, symmetric output and timing must all give the oracle's CSR bit for bit, and the
same results as direct launches."""
import os

import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu


def _context(graphs: bool):
    old = os.environ.get("RTG_GRAPHS")
    os.environ["RTG_GRAPHS"] = "1" if graphs else "0"
    try:
        return rtg.Context(0)
    finally:
        if old is None:
            os.environ.pop("RTG_GRAPHS", None)
        else:
            os.environ["RTG_GRAPHS"] = old


def _case(seed, n=9001, d=5, m=6, dtype=np.float64):
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(seed, n, d, dtype)
    T = gen.transforms(seed, d, m, r)
    return pts, r, T


@pytest.mark.parametrize("graphs", [True, False])
def test_repeated_shape_new_data(graphs):
    import torch
    ctx = _context(graphs)
    try:
        for k, seed in enumerate([40, 41, 42, 43, 44]):
            pts, r, T = _case(seed)
            arg = torch.from_numpy(pts).cuda() if k % 2 else pts
            res = ctx.all_pairs(arg, r, T, r, timing=(k == 3))
            rp, col = res.download()
            st = res.stats
            res.release()
            ref = oracle.rtg(pts, r, T, r)
            assert np.array_equal(rp, ref.csr.row_ptr) and np.array_equal(col, ref.csr.col)
            assert st["candidates"] == [s["candidates"] for s in ref.stats]
            assert st["near_wall"] == sum(s["near_wall"] for s in ref.stats)
            assert st["attempts"] == 1
            if k == 3:
                assert st["phase_us"]["total"] > 0 and st["phase_us"]["sort"] > 0
    finally:
        ctx.close()


def test_symmetric_and_fp32_shapes_interleaved():
    ctx = _context(True)
    try:
        for k in range(4):
            pts, r, T = _case(50 + k, n=7000, d=4, m=5, dtype=np.float32 if k % 2 else np.float64)
            res = ctx.all_pairs(pts, r, T, r, symmetric=True)
            rp, col = res.download()
            res.release()
            ref = oracle.rtg(pts, r, T, r)
            p = ref.csr.pairs()
            both = np.concatenate([p, p[:, ::-1]])
            both = both[np.lexsort((both[:, 1], both[:, 0]))]
            want_rp = np.zeros(len(pts) + 1, dtype=np.int64)
            np.add.at(want_rp, both[:, 0] + 1, 1)
            assert np.array_equal(rp, np.cumsum(want_rp))
            assert np.array_equal(col, both[:, 1].astype(np.int32))
    finally:
        ctx.close()


def test_pair_buffer_growth_falls_back_and_recaptures():
    # a shape whose second input has far more pairs: the guessed pair buffer overflows, the
    # build re-runs directly, and the next replay uses the grown buffer
    ctx = _context(True)
    try:
        n, d, m = 6000, 3, 4
        r = 0.05
        T = gen.transforms(60, d, m, r)
        sparse = gen.points_uniform(60, n, d)
        dense = gen.points_mixture(61, n, d, k=2, sigma=0.02, dtype=np.float64)
        for pts in (sparse, sparse, dense, dense, sparse):
            res = ctx.all_pairs(pts, r, T, r)
            rp, col = res.download()
            res.release()
            ref = oracle.rtg(pts, r, T, r)
            assert np.array_equal(rp, ref.csr.row_ptr) and np.array_equal(col, ref.csr.col)
    finally:
        ctx.close()
