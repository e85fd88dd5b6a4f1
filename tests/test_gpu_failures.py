"""Failure detection without a GPU fault: bounded device waits that run out return
RTG_E_TIMEOUT and leave the context usable; a failed device allocation returns RTG_E_NOMEM;
a host wait with a short limit returns RTG_E_TIMEOUT and the ticket still completes.

Each hook (rtg_set_test_hooks) only makes a bounded wait wait for something that never
happens, or one allocation give up: nothing traps, faults or hangs.  After every failure the
next build on the same context is compared element by element with the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu


def workload(n=100000, d=6, m=8, seed=0):
    pts = gen.points_uniform(seed, n, d)
    r = gen.radius_for_degree(n, d)
    T = gen.transforms(seed, d, m, r)
    return pts, r, T


_REF = {}


def reference(n=100000, d=6, m=8, seed=0):
    key = (n, d, m, seed)
    if key not in _REF:
        pts, r, T = workload(n, d, m, seed)
        _REF[key] = oracle.rtg(pts, r, T, r).csr
    return _REF[key]


def assert_exact(ctx, pts, r, T):
    res = ctx.all_pairs(pts, r, T, r)
    rp, col = res.download()
    res.release()
    ref = reference(pts.shape[0], pts.shape[1], len(T))
    assert np.array_equal(rp, ref.row_ptr)
    assert np.array_equal(col, ref.col)


@pytest.mark.parametrize("hook", [rtg.RTG_INJECT_SORT_WAIT, rtg.RTG_INJECT_SCAN_WAIT],
                         ids=["sort_lookback", "csr_scan"])
def test_bounded_wait_times_out_and_context_stays_usable(hook, monkeypatch):
    # the look-back sort strategy (the one with inter-block waits) for this context
    monkeypatch.setenv("RTG_SORT_VARIANT", "8,12,0")
    monkeypatch.setenv("RTG_AUTOTUNE", "0")
    pts, r, T = workload()
    with rtg.Context(0) as ctx:
        assert_exact(ctx, pts, r, T)  # the shape's launch plan (and graph) exists
        rtg.rtg_set_test_hooks(ctx.handle, hook, 64, 0)
        with pytest.raises(rtg.RTGError) as e:
            ctx.all_pairs(pts, r, T, r)
        assert e.value.status == rtg.RTG_E_TIMEOUT
        assert "wait" in rtg.lib().rtg_last_error(ctx.handle).decode()
        rtg.rtg_set_test_hooks(ctx.handle, 0, 0, 0)
        assert_exact(ctx, pts, r, T)
        assert_exact(ctx, pts, r, T)


def test_tensor_core_wait_times_out_and_context_stays_usable():
    import torch

    n, d = 5000, 6
    pts = gen.points_uniform(4, n, d)
    r = gen.radius_for_degree(n, d, 30.0)
    ref = oracle.brute(pts, r)
    dev = torch.from_numpy(pts).cuda()
    with rtg.Context(0) as ctx:
        rtg.rtg_set_test_hooks(ctx.handle, rtg.RTG_INJECT_TC_WAIT, 1024, 0)
        with pytest.raises(rtg.RTGError) as e:
            ctx.brute_force(dev, r, tensor="fp16")
        assert e.value.status == rtg.RTG_E_TIMEOUT
        rtg.rtg_set_test_hooks(ctx.handle, 0, 0, 0)
        res = ctx.brute_force(dev, r, tensor="fp16")
        rp, col = res.download()
        res.release()
        assert np.array_equal(rp, ref.row_ptr)
        assert np.array_equal(col, ref.col)


@pytest.mark.parametrize("after", [1, 2, 5])
def test_allocation_failure_returns_nomem(after):
    pts, r, T = workload()
    with rtg.Context(0) as ctx:
        # a fresh context: the first build allocates its workspace, then its outputs
        rtg.rtg_set_test_hooks(ctx.handle, 0, 0, after)
        with pytest.raises(rtg.RTGError) as e:
            ctx.all_pairs(pts, r, T, r)
        assert e.value.status == rtg.RTG_E_NOMEM
        assert_exact(ctx, pts, r, T)
        # a warm context: the next allocation is the output CSR's
        rtg.rtg_set_test_hooks(ctx.handle, 0, 0, 1)
        with pytest.raises(rtg.RTGError) as e:
            ctx.all_pairs(pts, r, T, r)
        assert e.value.status == rtg.RTG_E_NOMEM
        assert_exact(ctx, pts, r, T)


def test_host_wait_with_a_short_limit_times_out_and_the_ticket_completes():
    pts, r, T = workload()
    with rtg.Context(0) as ctx:
        ticket = rtg.rtg_submit(ctx.handle, pts, r, T, r)
        with pytest.raises(rtg.RTGError) as e:
            rtg.rtg_wait(ctx.handle, ticket, 1)
        assert e.value.status == rtg.RTG_E_TIMEOUT
        res = ctx.wait(ticket, -1, m=len(T))
        rp, col = res.download()
        res.release()
        ref = reference()
        assert np.array_equal(rp, ref.row_ptr)
        assert np.array_equal(col, ref.col)


def test_fp64_coordinates_beyond_the_fp32_range_are_decided_in_fp64():
    # points in the unit cube plus a few far beyond the FP32 range (two of them close to
    # each other); cells wide enough that every cell index fits a key
    rng = np.random.default_rng(9)
    base = rng.random((3000, 3))
    far = np.array([[1e39, 0.1, 0.2], [1e39, 0.15, 0.2], [-4e38, 0.5, 0.5], [0.3, 7e300, 0.1]])
    pts = np.concatenate([base[:1000], far, base[1000:]])
    r, c, m = 0.3, 1e301, 3
    T = gen.transforms(9, 3, m, c)
    ref = oracle.rtg(pts, r, T, c).csr
    assert ref.nnz > 0
    with rtg.Context(0) as ctx:
        res = ctx.all_pairs(pts, r, T, c)
        rp, col = res.download()
        st = res.stats
        res.release()
    assert np.array_equal(rp, ref.row_ptr)
    assert np.array_equal(col, ref.col)
    assert st["key_rechecks"] > 0 and st["dist_rechecks"] > 0
