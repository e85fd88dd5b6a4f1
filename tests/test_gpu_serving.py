"""The request server (rtg_submit / rtg_poll / rtg_wait): every served result equals the
oracle's and the result of the same request built alone; admission by memory budget."""
import threading

import numpy as np
import pytest

import oracle
from paper_1409_8112_gb300 import gen, rtg

pytestmark = pytest.mark.gpu


def _requests(count, seed, m=8):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        d = int(rng.choice([2, 3, 6, 9]))
        n = int(np.floor(np.exp(rng.uniform(np.log(50), np.log(20000)))))
        if k % 3 == 0:
            pts = gen.points_mixture(seed * 1000 + k, n, d, k=8, sigma=0.05, dtype=np.float32)
        else:
            pts = gen.points_uniform(seed * 1000 + k, n, d, np.float32)
        r = gen.radius_for_degree(max(n, 2), d)
        T = gen.transforms(seed * 1000 + k, d, m, r)
        out.append((pts, r, T, r))
    return out


def test_served_results_equal_alone_and_oracle():
    ctx = rtg.Context(0)
    reqs = _requests(40, 3)
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for k in range(lo, hi):
            pts, r, T, c = reqs[k]
            tickets[k] = ctx.submit(pts, r, T, c)

    threads = [threading.Thread(target=submit, args=(q * 10, q * 10 + 10)) for q in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for k, (pts, r, T, c) in enumerate(reqs):
        res = ctx.wait(tickets[k], m=8)
        rp, col = res.download()
        ref = oracle.rtg(pts, r, T, c).csr
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col), k
        assert res.stats["phase_us"]["total"] >= res.stats["phase_us"]["prep"]
        res.release()
        alone = ctx.all_pairs(pts, r, T, c)
        ra, ca = alone.download()
        assert np.array_equal(rp, ra) and np.array_equal(col, ca)
        alone.release()
    ctx.close()


def test_poll_unknown_and_timeout():
    ctx = rtg.Context(0)
    with pytest.raises(rtg.RTGError) as e:
        rtg.rtg_poll(ctx.handle, 12345)
    assert e.value.status == rtg.RTG_E_UNKNOWN_TICKET
    pts, r, T, c = _requests(1, 5)[0]
    t = ctx.submit(pts, r, T, c)
    got = None
    while got is None:
        got = ctx.poll(t, m=8)
    rp, col = got.download()
    ref = oracle.rtg(pts, r, T, c).csr
    assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
    with pytest.raises(rtg.RTGError) as e:
        rtg.rtg_poll(ctx.handle, t)  # taken already
    assert e.value.status == rtg.RTG_E_UNKNOWN_TICKET
    ctx.close()


def test_budget_admission():
    # 96 MiB: small requests are served; a clustered request whose pairs cannot fit fails
    # with RTG_E_BUDGET without disturbing the others
    ctx = rtg.Context(0, mem_budget_bytes=96 << 20)
    small = _requests(6, 7, m=4)
    big_pts = gen.points_mixture(11, 200000, 3, k=2, sigma=0.01, dtype=np.float32)
    big_r = 0.05
    big_T = gen.transforms(11, 3, 4, big_r)
    tickets = [ctx.submit(*small[0])]
    big = ctx.submit(big_pts, big_r, big_T, big_r)
    tickets += [ctx.submit(*q) for q in small[1:]]
    with pytest.raises(rtg.RTGError) as e:
        ctx.wait(big)
    assert e.value.status == rtg.RTG_E_BUDGET
    for k, tk in enumerate(tickets):
        res = ctx.wait(tk, m=4)
        rp, col = res.download()
        ref = oracle.rtg(*small[k]).csr
        assert np.array_equal(rp, ref.row_ptr) and np.array_equal(col, ref.col)
        res.release()
    ctx.close()
