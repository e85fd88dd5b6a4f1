"""Grid parameters for a target recall (Sec. III-A): the chosen (c, m) must reach the target
on the sample and m - 1 grids of the same size must not (the smallest m), both checked with
the CPU oracle; the grids are the documented prefix of one seeded generation."""
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


def _recall(pts, r, T, c, exact):
    return oracle.rtg(pts, r, T, c).csr.nnz / exact


@pytest.mark.parametrize("shift_only", [False, True])
def test_choice_reaches_target_and_is_minimal(ctx, shift_only):
    n, d, target = 12000, 3, 0.9
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(41, n, d)
    ch = ctx.tune_params(pts, r, target, seed=7, shift_only=shift_only)
    assert ch["sample_n"] == n  # below the sample size: the whole input
    ex = oracle.brute(pts, r).nnz
    assert ch["sample_exact"] == ex
    flags = gen.SHIFT_ONLY if shift_only else 0
    m, c = ch["m"], ch["cell_side"]
    assert c == pytest.approx(ch["c_factor"] * r)
    T = gen.transforms(7, d, m, c, flags)
    rec = _recall(pts, r, T, c, ex)
    assert rec == pytest.approx(ch["recall"], abs=1e-12)
    assert rec >= target
    if m > 1:
        assert _recall(pts, r, T[: m - 1], c, ex) < target
    assert ch["build_us"] > 0 and ch["candidates"] > 0


def test_prefix_sample_for_large_inputs(ctx):
    n, d = 40000, 2
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(42, n, d, np.float32)
    ch = ctx.tune_params(pts, r, 0.8, seed=3)
    assert ch["sample_n"] == 32768
    assert ch["sample_exact"] == oracle.brute(pts[:32768], r).nnz
    assert ch["recall"] >= 0.8


def test_unreachable_target_is_refused(ctx):
    pts = gen.points_uniform(43, 500, 2)
    with pytest.raises(rtg.RTGError):
        ctx.tune_params(pts, 0.05, 1.5)
