"""Host-side arithmetic of the benchmark's JSON line (no GPU): the algorithmic bytes of the
roofline phases, the DRAM-traffic lookup per workload and sort variant, and the whole-job
throughput of replicas."""
import bench


def test_phase_bytes_model():
    n, d, m, kb, passes, dpad, pairs = 100000, 6, 8, 4, 4, 8, 456724
    N = n * m
    pb = bench.phase_bytes(n, d, m, kb, passes, dpad, pairs)
    # 8-bit digits: counted by the key kernel, so no extra read of the keys
    assert pb["sort"] == passes * 2 * N * (kb + 4)
    assert pb["pairs"] == N * (kb + 4) + N * dpad * 4 + 8 * pairs
    # wider digits: a histogram kernel reads the keys once more
    pb11 = bench.phase_bytes(n, d, m, kb, 3, dpad, pairs, digit_bits=11)
    assert pb11["sort"] == N * kb + 3 * 2 * N * (kb + 4)


def test_traffic_lookup_by_workload_and_sort_variant():
    cfg = {"digit_bits": 8, "tile_keys": 3072, "lookback": 1}
    t = bench.ncu_traffic(100000, "fp64", "sort", cfg)
    assert isinstance(t, int) and t > 0
    # a variant that was not captured has no traffic figure
    assert bench.ncu_traffic(100000, "fp64", "sort", dict(cfg, tile_keys=2048)) is None
    assert bench.ncu_traffic(123, "fp64", "pairs", cfg) is None
    assert bench.ncu_traffic(100000, "fp64", "pairs", cfg) > 0


def test_whole_job_throughput_counts_every_replica():
    one = bench.job_throughput(1000, 10, 1, 5.0)
    assert one == 1000 * 10 / 0.005
    assert bench.job_throughput(1000, 10, 4, 5.0) == 4 * one
    assert bench.max_over_ranks(7.5, 1) == 7.5
