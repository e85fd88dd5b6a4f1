"""Pins that tie the CPU oracle to the paper and to mathematics, not to itself.

Each ``pin_*`` takes the oracle build to check (``mutant`` 0 is the real oracle; other
values are builds with one planted mistake) and raises AssertionError on a mismatch.
test_oracle.py runs them all on the real oracle; test_oracle_mutants.py checks that every
planted mistake is caught by at least one of them.
"""
import numpy as np

import oracle
from golden_io import load_table2, load_worked
from paper_1409_8112_gb300 import gen


def _pairset(csr):
    return {tuple(map(int, p)) for p in csr.pairs()}


def _check_csr_shape(csr, n):
    assert csr.n == n
    assert csr.row_ptr[0] == 0 and np.all(np.diff(csr.row_ptr) >= 0)
    rows = np.repeat(np.arange(n), np.diff(csr.row_ptr))
    assert np.all(csr.col > rows), "every stored column must exceed its row (i < j)"
    for i in range(n):
        seg = csr.col[csr.row_ptr[i]:csr.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0), "columns strictly ascending within a row"


def pin_worked_2d(mutant=0):
    """Hand-derived worked example (tests/golden/rtg_2d_worked.txt): cells, grid-0 pairs,
    two-grid pairs and the exact set."""
    g = load_worked("rtg_2d_worked.txt")
    q, _ = oracle.cells(g["points"], g["transforms"], g["c"], mutant=mutant)
    assert np.array_equal(q, g["cells"]), f"cells {q.tolist()} != {g['cells'].tolist()}"
    one = oracle.rtg(g["points"], g["r"], g["transforms"][:1], g["c"], mutant=mutant)
    assert _pairset(one.csr) == g["rtg_grid0"]
    both = oracle.rtg(g["points"], g["r"], g["transforms"], g["c"], mutant=mutant)
    assert _pairset(both.csr) == g["rtg"]
    assert _pairset(oracle.brute(g["points"], g["r"], mutant=mutant)) == g["exact"]
    assert _pairset(oracle.exact_grid(g["points"], g["r"], mutant=mutant)) == g["exact"]


def pin_worked_boundary(mutant=0):
    """Dyadic worked example (tests/golden/rtg_boundary_worked.txt): a pair at distance
    exactly r is reported, one 2^-40 beyond r^2 is not, all axes count, duplicates count."""
    g = load_worked("rtg_boundary_worked.txt")
    q, _ = oracle.cells(g["points"], g["transforms"], g["c"], mutant=mutant)
    assert np.array_equal(q, g["cells"])
    res = oracle.rtg(g["points"], g["r"], g["transforms"], g["c"], mutant=mutant)
    assert _pairset(res.csr) == g["rtg"], _pairset(res.csr)
    assert _pairset(oracle.brute(g["points"], g["r"], mutant=mutant)) == g["exact"]


def pin_exact_grid_equals_brute(mutant=0):
    """Two different algorithms for the exact set (all pairs vs the adjacent-cell grid of
    Sec. II-B) must agree on random inputs across dimensions."""
    for d, n in ((1, 400), (2, 600), (3, 800), (6, 600), (12, 300)):
        pts = gen.points_uniform(100 + d, n, d)
        r = gen.radius_for_degree(n, d, 8.0)
        a = oracle.brute(pts, r, mutant=mutant)
        b = oracle.exact_grid(pts, r, mutant=mutant)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col), d
        assert a.nnz > 0


def pin_single_cell_equals_brute(mutant=0):
    """Special case: a cell larger than the whole (rotated) point set, with the shift at
    half a cell, puts every point in one cell, so Alg. 1 reports exactly the exact set."""
    for d in (2, 3, 6):
        n = 500
        pts = gen.points_uniform(7 + d, n, d)
        r = gen.radius_for_degree(n, d, 10.0)
        c = 8.0 * np.sqrt(d)
        T = gen.transforms(3, d, 2, c)
        T[:, d * d:] = c / 2
        res = oracle.rtg(pts, r, T, c, mutant=mutant)
        ex = oracle.brute(pts, r, mutant=mutant)
        assert np.array_equal(res.csr.row_ptr, ex.row_ptr) and np.array_equal(res.csr.col, ex.col)
        assert all(s["nonempty_cells"] == 1 for s in res.stats)


def pin_invariants(mutant=0):
    """Structural facts of Alg. 1: i < j with ascending columns, no self-pairs, RTG is a
    subset of the exact set, the union over grids decomposes grid by grid, a prefix of the
    grids reports a subset (recall never falls as m grows), relabelling the points
    relabels the output, and duplicate points are always reported."""
    n, d, m = 1500, 3, 5
    pts = gen.points_uniform(11, n, d)
    pts[7] = pts[3]  # a duplicate pair
    r = gen.radius_for_degree(n, d, 12.0)
    T = gen.transforms(5, d, m, r)
    full = oracle.rtg(pts, r, T, r, mutant=mutant)
    _check_csr_shape(full.csr, n)
    exact = _pairset(oracle.brute(pts, r, mutant=mutant))
    got = _pairset(full.csr)
    assert got <= exact
    assert (3, 7) in got
    union = set()
    prev = set()
    for t in range(m):
        union |= _pairset(oracle.rtg(pts, r, T[t:t + 1], r, mutant=mutant).csr)
        pre = _pairset(oracle.rtg(pts, r, T[:t + 1], r, mutant=mutant).csr)
        assert prev <= pre
        prev = pre
    assert union == got
    assert prev == got
    perm = np.random.default_rng(0).permutation(n)
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    res_p = _pairset(oracle.rtg(pts[perm], r, T, r, mutant=mutant).csr)
    mapped = {tuple(sorted((int(inv[i]), int(inv[j])))) for (i, j) in got}
    assert res_p == mapped


def pin_shift_probability(mutant=0):
    """Closed form for shift-only grids: two points whose offset is delta share a cell with
    probability prod_k max(0, 1 - |delta_k| / c) over a uniform shift.  Checked over 10^4
    seeded grids within 4.5 binomial standard deviations."""
    trials = 10000
    for d, delta in ((1, [0.3]), (3, [0.2, 0.5, 0.1])):
        c = 1.0
        pts = np.zeros((2, d))
        pts[1] = delta
        T = gen.transforms(42 + d, d, trials, c, flags=gen.SHIFT_ONLY)
        q, _ = oracle.cells(pts, T, c, mutant=mutant)
        same = np.all(q[:, 0, :] == q[:, 1, :], axis=1).mean()
        p = float(np.prod([max(0.0, 1 - abs(x) / c) for x in delta]))
        sd = np.sqrt(p * (1 - p) / trials)
        assert abs(same - p) <= 4.5 * sd, (d, same, p)


def pin_table2_recall(mutant=0, rows=None):
    """Table II (Sec. IV-A): with the tabulated m and c~ (c = c~ r), shift-only grids and r
    from Eq. 2 in the unit d-cube, at least 98% of the neighbouring pairs are reported
    (mean over three seeded point sets)."""
    rows = rows if rows is not None else load_table2()[:2]
    for d, n, m, ct in rows:
        recalls = []
        for seed in range(3):
            pts = gen.points_uniform(1000 + seed, n, d)
            r = gen.radius_fmt(n, d)
            T = gen.transforms(2000 + seed, d, m, ct * r, flags=gen.SHIFT_ONLY)
            res = oracle.rtg(pts, r, T, ct * r, mutant=mutant)
            ex = oracle.exact_grid(pts, r, mutant=mutant)
            recalls.append(oracle.recall(res.csr, ex))
        assert np.mean(recalls) >= 0.98, (d, n, m, ct, recalls)


def pin_candidate_counts(mutant=0):
    """Per-grid candidate count sum_u C(|u|, 2) equals the number of index pairs i < j that
    share a cell, counted pair by pair from the cell coordinates."""
    n, d, m = 400, 2, 3
    pts = gen.points_uniform(21, n, d)
    r = 0.08
    T = gen.transforms(22, d, m, r)
    res = oracle.rtg(pts, r, T, r, mutant=mutant)
    q, _ = oracle.cells(pts, T, r, mutant=mutant)
    for t in range(m):
        same = np.all(q[t][:, None, :] == q[t][None, :, :], axis=2)
        want = int(np.triu(same, 1).sum())
        assert res.stats[t]["candidates"] == want
        assert res.stats[t]["nonempty_cells"] == len({tuple(x) for x in q[t]})


def pin_queries(mutant=0):
    """Queries of new points from the stored grids (Sec. V).  (1) With one cell larger than the
    whole point set the answer to a query is every point within r (numpy distances; pairs
    within 1e-9 r of r are left out of the comparison).  (2) Querying the points themselves
    gives each point plus its RTG neighbours, the symmetric form of Alg. 1's pair set.
    (3) Queries far outside the grids' occupied cells get no answer.  (4) Answers lie within
    r and a prefix of the grids answers a subset."""
    d, n = 3, 400
    pts = gen.points_uniform(21, n, d)
    r = gen.radius_for_degree(n, d, 10.0)
    qs = np.concatenate([gen.points_uniform(22, 60, d), pts[:20]])
    c = 8.0 * np.sqrt(d)
    T = gen.transforms(4, d, 2, c)
    T[:, d * d:] = c / 2
    res = oracle.rtg_query(pts, r, T, c, qs, mutant=mutant)
    assert res.n == len(qs)
    dist = np.sqrt(((qs[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    for k in range(len(qs)):
        got = set(map(int, res.col[res.row_ptr[k]:res.row_ptr[k + 1]]))
        sure = np.abs(dist[k] - r) > 1e-9 * r
        want = set(np.nonzero((dist[k] <= r) & sure)[0].tolist())
        assert {j for j in got if sure[j]} == want, k
    # (2) the points as queries
    m = 4
    T = gen.transforms(5, d, m, r)
    full = oracle.rtg(pts, r, T, r, mutant=mutant)
    nb = [{i} for i in range(n)]
    for (i, j) in _pairset(full.csr):
        nb[i].add(j)
        nb[j].add(i)
    res = oracle.rtg_query(pts, r, T, r, pts, mutant=mutant)
    for i in range(n):
        row = res.col[res.row_ptr[i]:res.row_ptr[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert set(map(int, row)) == nb[i], i
    # (3) far away
    far = oracle.rtg_query(pts, r, T, r, qs + 100.0, mutant=mutant)
    assert far.nnz == 0
    # (4) within r, and prefix-monotone in the grids
    prev = None
    for t in range(1, m + 1):
        cur = oracle.rtg_query(pts, r, T[:t], r, qs, mutant=mutant)
        rows = np.repeat(np.arange(len(qs)), np.diff(cur.row_ptr))
        assert np.all(dist[rows, cur.col] <= r * (1 + 1e-12))
        pairs = set(zip(rows.tolist(), cur.col.tolist()))
        if prev is not None:
            assert prev <= pairs
        prev = pairs


ALL_PINS = [pin_worked_2d, pin_worked_boundary, pin_exact_grid_equals_brute,
            pin_single_cell_equals_brute, pin_invariants, pin_shift_probability,
            pin_table2_recall, pin_candidate_counts, pin_queries]
