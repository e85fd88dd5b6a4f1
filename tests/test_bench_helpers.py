"""Host-side arithmetic of the benchmark's JSON line (no GPU): the algorithmic bytes of the
roofline phases, the DRAM-traffic lookup per workload and sort variant, the whole-job
throughput of replicas, and the clock samples kept for the timed window."""
import bench


def test_phase_bytes_model():
    n, d, m, kb, passes, pairs = 100000, 6, 8, 4, 4, 456724
    N = n * m
    # FP64 coordinates: the pairs model gathers d * 8 bytes per (point, grid) element
    pb = bench.phase_bytes(n, d, m, kb, passes, 8, pairs)
    assert pb["pairs"] == N * (kb + 4) + N * d * 8 + 8 * pairs
    # the first pass reads only the key rows; every pass writes keys and indices
    assert pb["sort"] == N * kb + N * (kb + 4) + (passes - 1) * 2 * N * (kb + 4)
    # a histogram kernel reads the keys once more
    pbh = bench.phase_bytes(n, d, m, kb, 3, 4, pairs, hist_read=True)
    assert pbh["sort"] == N * kb + N * kb + N * (kb + 4) + 2 * 2 * N * (kb + 4)
    assert pbh["pairs"] == N * (kb + 4) + N * d * 4 + 8 * pairs


def test_traffic_lookup_by_workload_and_sort_variant(monkeypatch):
    cfg = {"digit_bits": 8, "tile_keys": 3072, "lookback": 1, "passes": 4}
    monkeypatch.setattr(bench, "NCU_TRAFFIC",
                        {(100000, "fp64"): {"pairs": 123, "sort": {(8, 3072, 1, 4): 456}}})
    assert bench.ncu_traffic(100000, "fp64", "sort", cfg) == 456
    # a variant, or a pass count, that was not captured has no traffic figure
    assert bench.ncu_traffic(100000, "fp64", "sort", dict(cfg, tile_keys=2048)) is None
    assert bench.ncu_traffic(100000, "fp64", "sort", dict(cfg, passes=3)) is None
    assert bench.ncu_traffic(123, "fp64", "pairs", cfg) is None
    assert bench.ncu_traffic(100000, "fp64", "pairs", cfg) == 123


def test_whole_job_throughput_counts_every_replica():
    one = bench.job_throughput(1000, 10, 1, 5.0)
    assert one == 1000 * 10 / 0.005
    assert bench.job_throughput(1000, 10, 4, 5.0) == 4 * one
    assert bench.max_over_ranks(7.5, 1) == 7.5


def test_clock_samples_count_only_inside_the_timed_window():
    import time

    class Done:  # a finished nvidia-smi process
        def poll(self):
            return 0

        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    c = bench.ClockSampler(0)
    c.proc = Done()
    now = time.perf_counter()
    row = "0, {}, 2070, 800, 0x0, Not Active, Not Active, Not Active, {}"
    # a sample from the warm-up (clock low, power cap active) and two from the timed steps
    c.lines = [(now - 5.0, row.format(1200, "Active")), (now - 0.05, row.format(2070, "Not Active")),
               (now, row.format(2055, "Not Active"))]
    c.open_window()
    c.t_open = now - 0.1
    rec = c.stop()
    assert rec["samples"] == 2 and rec["reasons"] == [] and rec["sm_max_mhz"] == 2070.0
    assert 2055.0 <= rec["sm_mhz"] <= 2070.0
