"""Tensor-core brute force (tcgen05 tiles, FP16 / BF16 hi-lo split, FP32 accumulation, FP64
band check): the pair set equals the FP64 definition exactly, and the observed tile error
stays inside the band."""
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


@pytest.mark.parametrize("tensor", ["fp16", "bf16"])
@pytest.mark.parametrize("d,n,dtype", [(1, 700, np.float64), (3, 3001, np.float64),
                                       (6, 4099, np.float32), (9, 2500, np.float64),
                                       (16, 1300, np.float32)])
def test_tc_brute_matches_oracle(ctx, tensor, d, n, dtype):
    pts = gen.points_uniform(50 + d, n, d, dtype)
    r = gen.radius_for_degree(n, d, 20.0)
    res = ctx.brute_force(pts, r, tensor=tensor)
    rp, col = res.download()
    ex = oracle.brute(pts, r)
    assert np.array_equal(rp, ex.row_ptr) and np.array_equal(col, ex.col)
    st = res.stats
    assert st["band"] >= 1e-3 * r * r * (1 - 1e-12)
    assert st["max_abs_err_d2"] < st["band"]
    res.release()


def test_tc_offset_coordinates(ctx):
    pts = gen.points_uniform(8, 3000, 4) * 2.0 + 5.0  # centring keeps the split accurate
    r = 0.25
    for tensor in ("fp16", "bf16"):
        res = ctx.brute_force(pts, r, tensor=tensor)
        rp, col = res.download()
        ex = oracle.brute(pts, r)
        assert np.array_equal(rp, ex.row_ptr) and np.array_equal(col, ex.col)


@pytest.mark.parametrize("tensor", ["fp16", "bf16"])
@pytest.mark.parametrize("sigma,n,d,dtype", [(0.01, 6000, 3, np.float32),
                                             (0.02, 8000, 6, np.float64),
                                             (0.05, 9000, 6, np.float32),
                                             (0.05, 5000, 12, np.float32)])
def test_dense_cells_on_tensor_cores_match_oracle(ctx, tensor, sigma, n, d, dtype):
    # clustered points (8 Gaussians): cells of hundreds to thousands of points, whose pairs go
    # through the tensor-core tiles; the set must equal the oracle's and the build without
    # the tiles, candidate counts included
    pts = gen.points_mixture(70 + d, n, d, k=8, sigma=sigma, dtype=dtype)
    r = gen.radius_for_degree(n, d, 6.0)
    T = gen.transforms(70 + d, d, 4, r)
    res = ctx.all_pairs(pts, r, T, r, tensor=tensor)
    rp, col = res.download()
    st = res.stats
    res.release()
    ref = oracle.rtg(pts, r, T, r)
    assert np.array_equal(rp, ref.csr.row_ptr) and np.array_equal(col, ref.csr.col)
    assert st["candidates"] == [s["candidates"] for s in ref.stats]
    assert st["large_cells"] > 0 and st["max_cell"] > 256
