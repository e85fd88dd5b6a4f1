"""rtg_brute_count_noalloc (the entry point for callers that cannot allocate device memory,
e.g. a planner loop under a fixed memory plan) against rtg_brute_force's exact count.

Kept in a file of its own that pytest collects last, so a run that stops at the first
failure has already run every other test.  It must pass alone in a fresh process too."""
import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu


def test_noalloc_count_matches_brute_force_on_consecutive_calls():
    import torch

    stream = torch.cuda.current_stream()
    # calls in a row on different inputs, each against the existing entry point; every call
    # is smaller than the one before, so stale scratch from an earlier call would show.  The
    # first fills the static scratch to its limit (65536 points of 16 coordinates, the
    # widest FP32 rows).
    cases = [(65536, 16, np.float32, 3), (60000, 6, np.float64, 1), (9000, 3, np.float32, 2)]
    with rtg.Context(0) as ctx:
        for n, d, dt, seed in cases:
            pts = gen.points_uniform(seed, n, d, dt)
            r = gen.radius_for_degree(n, d, 12.0)
            dev = torch.from_numpy(pts).cuda()
            stream.synchronize()
            code = rtg.RTG_DTYPE_F64 if dt == np.float64 else rtg.RTG_DTYPE_F32
            got = rtg.rtg_brute_count_noalloc(dev.data_ptr(), code, n, d, r, stream.cuda_stream)
            ref = ctx.brute_force(dev, r, count_only=True)
            assert got == ref.nnz and got > 0
            ref.release()


def test_noalloc_rejects_sizes_beyond_the_static_limit():
    import torch

    dev = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(rtg.RTGError) as e:
        rtg.rtg_brute_count_noalloc(dev.data_ptr(), rtg.RTG_DTYPE_F64, 65537, 3, 0.1)
    assert e.value.status == rtg.RTG_E_INVALID
    assert "65536" in rtg.lib().rtg_last_error(None).decode()


def test_noalloc_count_matches_the_cpu_oracle():
    import torch

    # a small case against the CPU oracle's brute force (independent of the GPU kernels)
    n, d = 1500, 5
    pts = gen.points_uniform(11, n, d)
    r = gen.radius_for_degree(n, d, 20.0)
    dev = torch.from_numpy(pts).cuda()
    torch.cuda.synchronize()
    got = rtg.rtg_brute_count_noalloc(dev.data_ptr(), rtg.RTG_DTYPE_F64, n, d, r)
    assert got == oracle.brute(pts, r).nnz > 0


def test_noalloc_refuses_a_capturing_stream():
    import torch

    # the call synchronises its stream and reads the count back, so inside a capture it must
    # refuse before it issues anything (the capture itself stays valid)
    n, d = 2000, 4
    pts = gen.points_uniform(12, n, d)
    r = gen.radius_for_degree(n, d, 10.0)
    dev = torch.from_numpy(pts).cuda()
    side = torch.zeros(16, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = []
    with torch.cuda.graph(g, stream=s):
        side.add_(1.0)
        try:
            rtg.rtg_brute_count_noalloc(dev.data_ptr(), rtg.RTG_DTYPE_F64, n, d, r, s.cuda_stream)
            status.append(rtg.RTG_OK)
        except rtg.RTGError as e:
            status.append(e.status)
    g.replay()
    torch.cuda.synchronize()
    assert status == [rtg.RTG_E_INVALID]
    assert float(side[0]) == 1.0
    # outside the capture the same call counts as before
    got = rtg.rtg_brute_count_noalloc(dev.data_ptr(), rtg.RTG_DTYPE_F64, n, d, r)
    assert got == oracle.brute(pts, r).nnz > 0
