"""The CPU oracle against its pins (paper values, closed forms, invariants, brute force)."""
import numpy as np
import pytest

import oracle
import pins
from golden_io import load_table2
from paper_1409_8112_gb300 import gen


@pytest.mark.parametrize("pin", [p for p in pins.ALL_PINS if p is not pins.pin_table2_recall],
                         ids=lambda p: p.__name__)
def test_pin(pin):
    pin(0)


@pytest.mark.slow
@pytest.mark.parametrize("row", load_table2(), ids=lambda r: f"d{r[0]}_n{r[1]}")
def test_table2_recall(row):
    pins.pin_table2_recall(0, rows=[row])


def test_near_r_and_near_wall_diagnostics():
    # A pair exactly at distance r is within 1e-12 r of r; a point exactly on a cell wall
    # of a shift-only grid is within 1e-12 of that wall.
    pts = np.array([[0.0, 0.0], [0.375, 0.5], [0.125, 0.0625]], dtype=np.float64)
    T = np.array([[1.0, 0.0, 0.0, 1.0, 0.0, 0.0]])
    res = oracle.rtg(pts, 0.625, T, 1.0)
    assert res.near_r == 1
    # with c = 1/8 every point has a coordinate that is an exact multiple of c
    _, near = oracle.cells(pts, T, 0.125)
    assert near[0] == 3
    # shifted by c/4 on both axes, every coordinate sits a quarter cell from a wall
    T2 = np.array([[1.0, 0.0, 0.0, 1.0, 0.03125, 0.03125]])
    _, near2 = oracle.cells(pts, T2, 0.125)
    assert near2[0] == 0


def test_fp32_input_is_widened_exactly():
    p64 = gen.points_uniform(3, 300, 3)
    p32 = p64.astype(np.float32)
    r = 0.15
    T = gen.transforms(4, 3, 3, r)
    a = oracle.rtg(p32, r, T, r).csr
    b = oracle.rtg(p32.astype(np.float64), r, T, r).csr
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)


def test_empty_and_single_point():
    for n in (0, 1):
        pts = np.zeros((n, 3))
        T = gen.transforms(1, 3, 2, 0.1)
        res = oracle.rtg(pts, 0.1, T, 0.1)
        assert res.csr.nnz == 0 and len(res.csr.row_ptr) == n + 1


def test_transforms_are_haar_orthogonal():
    # Orthogonality, |det| = 1, shifts in [0, c), and the Haar moments of O(d):
    # E[tr R] = 0, E[tr(R)^2] = 1 (d >= 2), E[R_00^2] = 1/d.
    for d in (2, 3, 6, 9, 12):
        T = gen.transforms(77, d, 4000, 0.5)
        R = T[:, :d * d].reshape(-1, d, d)
        s = T[:, d * d:]
        err = np.abs(np.einsum("tki,tkj->tij", R, R) - np.eye(d)).max()
        assert err <= 1e-14
        assert np.allclose(np.abs(np.linalg.det(R)), 1.0, atol=1e-12)
        assert s.min() >= 0.0 and s.max() < 0.5
        tr = np.trace(R, axis1=1, axis2=2)
        assert abs(tr.mean()) < 5 * 1.0 / np.sqrt(4000)
        assert abs((tr ** 2).mean() - 1.0) < 0.15
        assert abs((R[:, 0, 0] ** 2).mean() - 1.0 / d) < 0.05 / np.sqrt(d)


def test_shift_only_flag_gives_identity():
    T = gen.transforms(1, 4, 3, 0.2, flags=gen.SHIFT_ONLY)
    for t in range(3):
        assert np.array_equal(T[t, :16].reshape(4, 4), np.eye(4))


def test_radius_for_expected_degree():
    # r^d * zeta_d * n = 2 ln n, with zeta_6 = pi^3 / 6; for n = 1e5, d = 6, r = 0.188287.
    r = gen.radius_for_degree(100000, 6)
    assert abs(r - 0.18829) < 1e-5
    assert abs(r ** 6 * np.pi ** 3 / 6 * 100000 - 2 * np.log(100000)) < 1e-9


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_oracle_equals_serial(threads):
    # The all-core CPU baseline runs oracle_rtg_threads: grids on several threads, the merge
    # split by row ranges.  It must give the serial oracle's CSR exactly, including a case
    # with more threads than grids and rows.
    for seed, n, d, m, c_mul in [(0, 3000, 3, 5, 1.0), (1, 2000, 6, 8, 1.3), (2, 5, 2, 4, 1.0)]:
        pts = gen.points_uniform(seed, n, d)
        r = gen.radius_for_degree(max(n, 2), d)
        T = gen.transforms(seed, d, m, c_mul * r)
        a = oracle.rtg(pts, r, T, c_mul * r).csr
        b = oracle.rtg_threads(pts, r, T, c_mul * r, threads)
        assert np.array_equal(a.row_ptr, b.row_ptr)
        assert np.array_equal(a.col, b.col)
