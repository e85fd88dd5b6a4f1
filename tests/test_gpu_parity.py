"""GPU library vs the CPU oracle, element by element, through the C ABI.

The bar is bit-exact equality of the CSR (row pointers and columns) and of the exact
integer statistics (per-grid candidate counts, largest cell, near-wall and near-r counts)."""
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


def symmetric_of(csr, n):
    """Both (i, j) and (j, i) of every pair of an upper-triangular CSR, rows ascending."""
    p = csr.pairs()
    both = np.concatenate([p, p[:, ::-1]])
    both = both[np.lexsort((both[:, 1], both[:, 0]))]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, both[:, 0] + 1, 1)
    return np.cumsum(rp), both[:, 1].astype(np.int32)


def run_and_compare(ctx, pts, r, T, c, symmetric=False, on_device=False, check_stats=True):
    arg = pts
    if on_device:
        import torch
        arg = torch.from_numpy(pts).cuda()
    res = ctx.all_pairs(arg, r, T, c, symmetric=symmetric)
    rp, col = res.download()
    ref = oracle.rtg(pts, r, T, c)
    want_rp, want_col = ref.csr.row_ptr, ref.csr.col
    if symmetric:
        want_rp, want_col = symmetric_of(ref.csr, len(pts))
    assert len(rp) == len(want_rp)
    assert np.array_equal(rp, want_rp), "row pointers differ"
    assert np.array_equal(col, want_col), "columns differ"
    st = res.stats
    if check_stats:
        m = len(ref.stats)
        assert st["candidates"] == [s["candidates"] for s in ref.stats]
        assert st["max_cell"] == max(s["max_cell"] for s in ref.stats)
        assert st["near_wall"] == sum(s["near_wall"] for s in ref.stats)
        assert st["near_r"] == ref.near_r
        assert st["pairs"] == ref.csr.nnz
        assert len(st["candidates"]) == m
    res.release()
    return st, ref


def test_config1_n2000_d3(ctx):
    pts = gen.points_uniform(0, 2000, 3)
    T = gen.transforms(0, 3, 5, 0.1)
    st, ref = run_and_compare(ctx, pts, 0.1, T, 0.1)
    assert ref.csr.nnz > 4000


def test_config2_n100k_d6(ctx):
    n, d, m = 100000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(0, n, d)
    T = gen.transforms(0, d, m, r)
    st, ref = run_and_compare(ctx, pts, r, T, r)
    assert ref.csr.nnz > 400000


def test_config2_points_on_device_and_symmetric(ctx):
    n, d, m = 20000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(3, n, d)
    T = gen.transforms(3, d, m, r)
    run_and_compare(ctx, pts, r, T, r, on_device=True)
    run_and_compare(ctx, pts, r, T, r, symmetric=True, check_stats=False)


def test_fp32_points(ctx):
    n, d, m = 200000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(1, n, d, np.float32)
    T = gen.transforms(1, d, m, r)
    run_and_compare(ctx, pts, r, T, r)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 8, 9, 12, 16])
def test_dimensions(ctx, d):
    n = 3001
    r = gen.radius_for_degree(n, d, 10.0)
    pts = gen.points_uniform(10 + d, n, d)
    T = gen.transforms(20 + d, d, 4, 1.3 * r)
    run_and_compare(ctx, pts, r, T, 1.3 * r)


@pytest.mark.parametrize("m", [1, 2, 7, 64])
def test_grid_counts(ctx, m):
    n, d = 5000, 3
    r = gen.radius_for_degree(n, d, 12.0)
    pts = gen.points_uniform(5, n, d)
    T = gen.transforms(6, d, m, r)
    run_and_compare(ctx, pts, r, T, r)


def test_many_grids_high_dimension(ctx):
    # 64 grids of 16-dimensional rows: the key kernel's table of axis rows is too large to stage
    # the key rows in shared memory as well, so they go straight to global memory
    n, d, m = 3000, 16, 64
    r = gen.radius_for_degree(n, d, 10.0)
    pts = gen.points_uniform(7, n, d)
    T = gen.transforms(8, d, m, 1.2 * r)
    st, ref = run_and_compare(ctx, pts, r, T, 1.2 * r)
    assert ref.csr.nnz > 0


@pytest.mark.parametrize("symmetric", [False, True])
def test_rows_of_thousands_of_entries(ctx, symmetric):
    # every pair within r: rows of up to n - 1 entries take the block radix row sort
    n, d = 3000, 3
    pts = gen.points_uniform(14, n, d) * 0.01
    T = gen.transforms(15, d, 2, 0.1)
    st, ref = run_and_compare(ctx, pts, 0.1, T, 0.1, symmetric=symmetric)
    assert ref.csr.nnz == n * (n - 1) // 2


def test_download_into_caller_arrays(ctx):
    import torch
    pts = gen.points_uniform(12, 4000, 3)
    r = gen.radius_for_degree(4000, 3, 10.0)
    T = gen.transforms(13, 3, 4, r)
    res = ctx.all_pairs(pts, r, T, r)
    rp, col = res.download()
    bufs = (torch.empty(5000, dtype=torch.int64).pin_memory().numpy(),
            torch.empty(res.nnz + 100, dtype=torch.int32).pin_memory().numpy())
    rp2, col2 = res.download(bufs)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    with pytest.raises(ValueError):
        res.download((np.empty(10, dtype=np.int64), np.empty(res.nnz, dtype=np.int32)))
    res.release()


def test_shift_only_table2_parameters(ctx):
    n, d, m, ct = 12800, 3, 20, 1.15
    r = gen.radius_fmt(n, d)
    pts = gen.points_uniform(1000, n, d)
    T = gen.transforms(2000, d, m, ct * r, flags=gen.SHIFT_ONLY)
    run_and_compare(ctx, pts, r, T, ct * r)


def test_clustered_points_use_large_cells(ctx):
    # a Gaussian mixture with sigma well below the cell side gives cells of hundreds of points
    n, d, m = 20000, 3, 4
    pts = gen.points_mixture(9, n, d, k=4, sigma=0.01, dtype=np.float64)
    r = 0.05
    T = gen.transforms(9, d, m, r)
    st, ref = run_and_compare(ctx, pts, r, T, r)
    assert st["large_cells"] > 0 and st["max_cell"] > 128


def test_all_points_identical(ctx):
    pts = np.full((700, 4), 0.3)
    T = gen.transforms(2, 4, 3, 0.1)
    st, ref = run_and_compare(ctx, pts, 0.1, T, 0.1)
    assert ref.csr.nnz == 700 * 699 // 2


def test_single_cell_equals_brute_force(ctx):
    n, d = 3000, 3
    pts = gen.points_uniform(4, n, d)
    c = 8.0 * np.sqrt(d)
    T = gen.transforms(4, d, 2, c)
    T[:, d * d:] = c / 2
    r = 0.08
    res = ctx.all_pairs(pts, r, T, c)
    rp, col = res.download()
    ex = oracle.brute(pts, r)
    assert np.array_equal(rp, ex.row_ptr) and np.array_equal(col, ex.col)


def test_wide_keys_use_64_bits(ctx):
    n, d, m = 4000, 6, 3
    pts = gen.points_uniform(8, n, d)
    r = 0.02
    T = gen.transforms(8, d, m, r)
    st, _ = run_and_compare(ctx, pts, r, T, r)
    assert st["key_bits"] > 32


def test_offset_and_negative_coordinates(ctx):
    n, d = 8000, 4
    pts = gen.points_uniform(12, n, d) * 3.0 - 17.5
    r = 0.3
    T = gen.transforms(12, d, 5, 1.2 * r)
    run_and_compare(ctx, pts, r, T, 1.2 * r)


def test_walls_and_exact_radius_go_through_fp64(ctx):
    # dyadic points on a 1/8 lattice: every coordinate lies on a wall of the shift-only
    # grid with zero shift, and many pairs are exactly at distance r = 0.625
    g = np.arange(0, 1, 0.125)
    pts = np.array(np.meshgrid(g, g, g)).reshape(3, -1).T.copy()
    T = np.array([[1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]], dtype=np.float64)
    T = np.concatenate([T, gen.transforms(3, 3, 2, 0.625)])
    st, ref = run_and_compare(ctx, pts, 0.625, T, 0.625)
    assert st["near_wall"] > 0 and st["near_r"] > 0


def test_empty_and_tiny_inputs(ctx):
    T = gen.transforms(1, 3, 2, 0.1)
    for n in (0, 1, 2, 3, 33):
        pts = gen.points_uniform(n, n, 3) * 0.05
        run_and_compare(ctx, pts, 0.1, T, 0.1)


def test_errors(ctx):
    T = gen.transforms(1, 3, 2, 0.1)
    pts = gen.points_uniform(0, 100, 3)
    bad = pts.copy()
    bad[5, 1] = np.nan
    with pytest.raises(rtg.RTGError) as e:
        ctx.all_pairs(bad, 0.1, T, 0.1)
    assert e.value.status == rtg.RTG_E_INVALID
    with pytest.raises(rtg.RTGError) as e:
        ctx.all_pairs(pts, -0.1, T, 0.1)
    assert e.value.status == rtg.RTG_E_INVALID
    d = 16
    T16 = gen.transforms(1, d, 2, 1e-3)
    with pytest.raises(rtg.RTGError) as e:
        ctx.all_pairs(gen.points_uniform(0, 100, d), 1e-3, T16, 1e-3)
    assert e.value.status == rtg.RTG_E_KEY_OVERFLOW
    # the context stays usable after every error
    run_and_compare(ctx, pts, 0.1, T, 0.1)


def test_budget():
    small = rtg.Context(0, mem_budget_bytes=1 << 20)
    pts = gen.points_uniform(0, 20000, 3)
    T = gen.transforms(1, 3, 4, 0.05)
    with pytest.raises(rtg.RTGError) as e:
        small.all_pairs(pts, 0.05, T, 0.05)
    assert e.value.status == rtg.RTG_E_BUDGET
    small.close()


def test_repeatable(ctx):
    n, d = 30000, 6
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(2, n, d)
    T = gen.transforms(2, d, 8, r)
    a = ctx.all_pairs(pts, r, T, r).download()
    b = ctx.all_pairs(pts, r, T, r).download()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("d,n", [(1, 2000), (3, 3001), (6, 4099), (12, 2500)])
def test_brute_force_matches_oracle(ctx, d, n):
    pts = gen.points_uniform(40 + d, n, d)
    r = gen.radius_for_degree(n, d, 15.0)
    res = ctx.brute_force(pts, r)
    rp, col = res.download()
    ex = oracle.brute(pts, r)
    assert np.array_equal(rp, ex.row_ptr) and np.array_equal(col, ex.col)
    assert res.stats["pairs"] == ex.nnz


def test_brute_force_count_config2_and_recall(ctx):
    n, d, m = 100000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(0, n, d)
    cnt = ctx.brute_force(pts, r, count_only=True)
    ex = oracle.exact_grid(pts, r)
    assert cnt.nnz == ex.nnz
    T = gen.transforms(0, d, m, r)
    res = ctx.all_pairs(pts, r, T, r)
    assert 0.5 < res.nnz / cnt.nnz < 0.6


def _check_block(rp, col, lo, hi, ref):
    sub_rp = rp[lo:hi + 1] - rp[lo]
    sub_col = col[rp[lo]:rp[hi]] - lo
    assert np.array_equal(sub_rp, ref.row_ptr), "row pointers of an instance differ"
    assert np.array_equal(sub_col, ref.col), "columns of an instance differ"


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_batch_matches_each_instance(ctx, dtype):
    rng = np.random.default_rng(5)
    inst = []
    for b in range(14):
        d = [2, 3, 6, 9][b % 4]
        n = [0, 1, 2][b] if b < 3 else int(rng.integers(50, 4000))
        pts = gen.points_uniform(100 + b, n, d, dtype)
        r = gen.radius_for_degree(max(n, 2), d)
        T = gen.transforms(200 + b, d, 4, 1.1 * r)
        inst.append((pts, r, T, 1.1 * r))
    res, offs = ctx.batch_all_pairs(inst, m=4)
    rp, col = res.download()
    total = 0
    for b, (pts, r, T, c) in enumerate(inst):
        ref = oracle.rtg(pts, r, T, c).csr
        _check_block(rp, col, offs[b], offs[b + 1], ref)
        total += ref.nnz
    assert res.nnz == total
    res.release()


def test_batch_on_device_and_symmetric(ctx):
    import torch
    inst, host = [], []
    for b in range(6):
        n, d = 1500 + 300 * b, 3
        pts = gen.points_uniform(300 + b, n, d)
        r = gen.radius_for_degree(n, d)
        T = gen.transforms(400 + b, d, 5, r)
        inst.append((torch.from_numpy(pts).cuda(), r, T, r))
        host.append((pts, r, T, r))
    res, offs = ctx.batch_all_pairs(inst, m=5)
    rp, col = res.download()
    for b, (pts, r, T, c) in enumerate(host):
        _check_block(rp, col, offs[b], offs[b + 1], oracle.rtg(pts, r, T, c).csr)
    res.release()
    res, offs = ctx.batch_all_pairs(inst, m=5, symmetric=True)
    assert res.nnz == 2 * sum(oracle.rtg(p, r, T, c).csr.nnz for p, r, T, c in host)
    res.release()


def test_two_pass_mode_matches(ctx):
    n, d, m = 30000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(6, n, d)
    T = gen.transforms(6, d, m, r)
    a = ctx.all_pairs(pts, r, T, r, two_pass=True)
    ra, ca = a.download()
    ref = oracle.rtg(pts, r, T, r).csr
    assert np.array_equal(ra, ref.row_ptr) and np.array_equal(ca, ref.col)


@pytest.mark.parametrize("symmetric,timing", [(False, False), (True, False), (False, True)])
def test_launch_assumptions_are_corrected(symmetric, timing):
    # same shape, far more pairs (and dense cells) the second time: the build runs again with
    # the corrected launch decisions; the next build of the shape takes them at once
    ctx = rtg.Context(0)
    n, d, m = 6000, 3, 4
    r = 0.05
    T = gen.transforms(7, d, m, r)
    a = gen.points_uniform(7, n, d)
    b = gen.points_mixture(7, n, d, k=2, sigma=0.01, dtype=np.float64)
    ref = oracle.rtg(b, r, T, r).csr
    want = symmetric_of(ref, n) if symmetric else (ref.row_ptr, ref.col)
    ra = ctx.all_pairs(a, r, T, r, symmetric=symmetric)
    for k in range(2):
        rb = ctx.all_pairs(b, r, T, r, symmetric=symmetric, timing=timing)
        # the first build of b runs again with the dense-cell kernels (which a uniform build
        # of the shape left out), and may then recover an undersized pair buffer
        assert rb.stats["attempts"] in (2, 3) if k == 0 else rb.stats["attempts"] == 1
        got = rb.download()
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
        assert rb.stats["pairs"] == ref.nnz
        rb.release()
    ra.release()
    ctx.close()


@pytest.mark.parametrize("symmetric", [False, True])
def test_overflowed_pair_buffer_is_recovered_without_a_rebuild(symmetric):
    # a shape first built on clustered points (its dense-cell kernels stay in the launch), then
    # on denser clustered points: only the pair buffer is too small, so the rows counted by the
    # enumeration are placed and a second enumeration writes the columns into them
    ctx = rtg.Context(0)
    n, d, m = 6000, 3, 4
    r = 0.05
    T = gen.transforms(8, d, m, r)
    a = gen.points_mixture(8, n, d, k=2, sigma=0.02, dtype=np.float64)
    b = gen.points_mixture(9, n, d, k=2, sigma=0.006, dtype=np.float64)
    ref = oracle.rtg(b, r, T, r).csr
    want = symmetric_of(ref, n) if symmetric else (ref.row_ptr, ref.col)
    ra = ctx.all_pairs(a, r, T, r, symmetric=symmetric)
    assert ra.stats["large_cells"] > 0
    rb = ctx.all_pairs(b, r, T, r, symmetric=symmetric)
    assert rb.stats["attempts"] == 2 and rb.stats["pairs"] > 2 * ra.stats["pairs"]
    got = rb.download()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    ra.release()
    rb.release()
    ctx.close()


def test_kernels_left_out_come_back_when_work_turns_up():
    # uniform points leave the dense-cell kernels and the queued row sorts out of the next
    # build of the shape; clustered points of that shape bring them back (the kernels before
    # them flag the work and the build runs again), and the result is exact either way
    ctx = rtg.Context(0)
    n, d, m = 20000, 3, 4
    r = 0.02
    T = gen.transforms(10, d, m, r)
    u = gen.points_uniform(10, n, d)
    c = gen.points_mixture(10, n, d, k=2, sigma=0.01, dtype=np.float64)
    for pts, first in ((u, True), (u, False), (c, False), (c, False), (u, False)):
        res = ctx.all_pairs(pts, r, T, r)
        got = res.download()
        st = res.stats
        res.release()
        ref = oracle.rtg(pts, r, T, r).csr
        assert np.array_equal(got[0], ref.row_ptr) and np.array_equal(got[1], ref.col)
        if pts is u and not first:
            assert st["max_cell"] <= 24
    ctx.close()


@pytest.mark.parametrize("flags,ct", [(0, 1.1), (0, 1.6), (gen.SHIFT_ONLY, 1.35)])
def test_cells_wider_than_r_use_parity_signatures(ctx, flags, ct):
    # c well above r: the earlier-grid test of the medium and large cells runs on cell-parity
    # signatures; clustered points make many such cells
    n, d, m = 12000, 4, 12
    pts = np.concatenate([gen.points_uniform(81, n // 2, d),
                          gen.points_mixture(82, n - n // 2, d, k=3, sigma=0.03,
                                             dtype=np.float64)])
    r = gen.radius_for_degree(n, d)
    T = gen.transforms(83, d, m, ct * r, flags=flags)
    st, ref = run_and_compare(ctx, pts, r, T, ct * r)
    assert st["large_cells"] > 0
