"""Throughput of the RTG all-pairs r-NN build on GB300 (one JSON line on stdout).

Workload (the configuration the metric is quoted on): n = 100,000 points i.i.d. uniform in
[0,1]^6 stored FP64, r for an expected ball population of 2 ln n (r = 0.18829), m = 8 seeded
random rotations + shifts, cell side c = r, seed 0.  One step = one complete build: all m
grids keyed, grouped, enumerated, deduplicated and assembled into the device CSR.

  value : unique reported pairs per second of device time, points resident in HBM, L2
          flushed between steps (512 MB write, then a 256 MB read)
  e2e   : the same metric through the C ABI with host buffers: points copied in from pinned
          host memory and the CSR copied back into pinned host arrays (allocated once)
          inside the timed region
  --impl reference : the CPU oracle (test infrastructure) timed on the host cores on the
          same workload
Multi-GPU (torchrun): replicas only; every rank builds its own roadmap, no collective on
the data path; value = pairs of all ranks / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reported r-NN pairs/s and roadmap builds/s at recall R; p50/p99 build latency"
L2_FLUSH_BYTES = 512 << 20
L2_CLEAN_BYTES = 256 << 20
L2_NOTE = ("flushed between steps: 512 MB write, then a 256 MB read so that no dirty line of "
           "the flush buffer is written back inside the timed region")


class L2Flush:
    """Evicts the inputs from the 129 MB L2 before each timed step: a 512 MB write, then a
    256 MB read, so that the L2 holds only clean lines of an unrelated buffer."""

    def __init__(self):
        import torch
        self.buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
        self.clean = torch.zeros(L2_CLEAN_BYTES // 4, dtype=torch.int32, device="cuda")
        # first use outside any timed region: the fill and sum kernels load (and, where the
        # installed torch has no code for this GPU, compile) on first launch, which took
        # about 1.7 s of host time in the first process on a machine
        self(0)
        torch.cuda.synchronize()

    def __call__(self, k: int = 0):
        self.buf.fill_(k & 0xff)
        self.sink = self.clean.sum()


WORKLOAD = {"workload": "rtg_all_pairs n=100000 d=6 fp64 uniform[0,1]^6 r=2lnn-degree m=8 c=r seed0",
            "n": 100000, "d": 6, "m": 8, "points": "uniform [0,1]^6, fp64", "cell_side": "r",
            "seed": 0, "l2": L2_NOTE}



def set_workload(n: int, dtype: str):
    """The single-roadmap workload: n uniform points in [0,1]^6, m = 8, c = r for degree
    2 ln n, seed 0; FP64 (the headline, n = 100,000) or FP32 (the 1,000,000-point case)."""
    WORKLOAD["n"] = n
    WORKLOAD["points"] = f"uniform [0,1]^6, {dtype}"
    WORKLOAD["workload"] = (f"rtg_all_pairs n={n} d=6 {dtype} uniform[0,1]^6 r=2lnn-degree m=8 "
                            "c=r seed0")
    WORKLOAD["dtype"] = dtype


def workload():
    from paper_1409_8112_gb300 import gen
    n, d, m = WORKLOAD["n"], WORKLOAD["d"], WORKLOAD["m"]
    r = gen.radius_for_degree(n, d)
    pts = gen.points_uniform(0, n, d, np.float32 if WORKLOAD.get("dtype") == "fp32" else np.float64)
    T = gen.transforms(0, d, m, r)
    return pts, T, r


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(total_ms: float, ws: int, device="cuda") -> float:
    """Duration of the timed region for the whole job: the slowest replica decides (an
    all-reduce MAX over the ranks' own timings; the identity on one rank)."""
    if ws == 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pairs_per_build: int, steps: int, ws: int, total_ms: float) -> float:
    """Whole-job pairs/s: every rank builds `steps` roadmaps (replicas, weak scaling)."""
    return pairs_per_build * steps * ws / (total_ms / 1e3)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        """Starts sampling and returns once the first sample is in (at most 10 s): the first
        nvidia-smi call on a fresh machine initialises NVML and has stalled CUDA calls for
        over a second, which must not fall into the timed steps."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
            return
        t_end = time.perf_counter() + 10.0
        while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def open_window(self):
        """The timed region starts: samples from here (less one period) to stop() count."""
        self.t_open = time.perf_counter()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        t0 = getattr(self, "t_open", None)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in self.lines:
            if t0 is not None and t < t0 - 0.2:
                continue
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Algorithmic bytes per build of the two phases a roofline is reported for:
#   pairs : the survey's per-grid model of in-cell enumeration, summed over the m grids:
#           the sorted (key, index) of every (point, grid) element, a gather of each point's
#           coordinates in the input's own width (d * S bytes), and 8 bytes per emitted pair
#           (each reported pair is emitted once, by its first grid)
#   sort  : every radix pass reads and writes the N (key, index) elements (the first pass
#           reads the key rows only: indices are implicit), plus one read of the keys by a
#           histogram kernel when the key kernel did not count the digits
# DRAM bytes (read + write) of each phase's kernels per build, from ncu, for the profiled
# workloads and, for the sort, the variant the profiled run used (digit bits, keys per tile,
# look-back code).  None where the kernels changed after the capture.
NCU_TRAFFIC = {
    # DRAM bytes of the dominant kernel from one ncu capture, per workload; an entry goes when
    # its kernel changes.  pairs: k_pairs_warp, one launch; sort: the k_sort_pass launches of
    # one sort, per (digit bits, tile keys, look-back, passes).  The captures of both (13.2 MB
    # and 331.5 MB for the pairs at 100k and 1M, 24.2 MB for the four-pass 100k sort) predate
    # the cell-major sort, which changed k_pairs_warp and the sort's order at 100k.
}


def phase_bytes(n, d, m, key_bytes, passes, coord_bytes, pairs, hist_read=False):
    N = n * m
    return {
        "sort": (N * key_bytes if hist_read else 0) + N * key_bytes + N * (key_bytes + 4) +
                max(0, passes - 1) * 2 * N * (key_bytes + 4),
        "pairs": N * (key_bytes + 4) + N * d * coord_bytes + 8 * pairs,
    }


def ncu_traffic(n, dtype, phase, sort_cfg):
    t = NCU_TRAFFIC.get((n, dtype), {}).get(phase)
    if phase == "sort" and isinstance(t, dict):
        t = t.get((sort_cfg.get("digit_bits"), sort_cfg.get("tile_keys"), sort_cfg.get("lookback"),
                   sort_cfg.get("passes")))
    return t


def measure_build(ctx, stream, flush, args, pts, T, r, dtype_name, ws, rank, clocks=None):
    """Device-timed builds (inputs resident), their phases and roofline, and the end-to-end
    rate through the C ABI with host points and a CSR download.  Returns the fields of a
    bench record."""
    import torch
    import torch.distributed as dist
    n, d = pts.shape
    m = T.shape[0]
    dev_pts = torch.from_numpy(pts).cuda()
    if clocks is not None:
        clocks.start()  # sampling runs from before the warm-up; only the timed window counts
    # recall against the exact set (device brute force), outside the timed region
    exact = ctx.brute_force(dev_pts, r, count_only=True)
    exact_pairs = exact.nnz
    exact.release()
    for k in range(args.warmup):
        for timing in (False, True):  # both launch plans (with and without phase events)
            # the same calls as a timed step (flush, events, build, read-back), untimed
            flush(k)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = ctx.all_pairs(dev_pts, r, T, r, timing=timing)
            e1.record(stream)
            e1.synchronize()
            e0.elapsed_time(e1)
            res.stats
            res.release()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    if clocks is not None:
        clocks.open_window()

    def steps(timing):
        out_ms, out_ph, info = [], [], {}
        for k in range(args.steps):
            flush(k)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = ctx.all_pairs(dev_pts, r, T, r, timing=timing)
            e1.record(stream)
            e1.synchronize()
            out_ms.append(e0.elapsed_time(e1))
            st = res.stats
            if timing:
                out_ph.append(st["phase_us"])
            info = {"pairs": res.nnz, "launches": st["launches"], "key_bits": st["key_bits"],
                    "passes": st["sort_passes"], "sort": st["sort"],
                    "phase_bytes": st["phase_bytes"], "enumeration": st["enumeration"]}
            res.release()
        return out_ms, out_ph, info

    # timed region: whole builds, no instrumentation
    t_wall = time.perf_counter()
    step_ms, _, info = steps(False)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    wall_s = time.perf_counter() - t_wall
    # the same steps again with phase events (they cost about 30 us a build), for the roofline
    _, phases, _ = steps(True)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    pairs, launches = info["pairs"], info["launches"]
    key_bytes = 8 if info["key_bits"] > 32 else 4
    passes = info["passes"]
    sort_cfg = dict(info["sort"], key_bits=info["key_bits"], passes=passes)
    total_ms = max_over_ranks(float(np.sum(step_ms)), ws)
    ms_per_step = total_ms / args.steps

    # end to end through the C ABI with host buffers (pinned) and the CSR copied back
    host_pts = torch.from_numpy(pts).pin_memory()
    # pinned result buffers, reused by every step (the download is then a direct DMA)
    host_rp = torch.empty(n + 1, dtype=torch.int64).pin_memory().numpy()
    host_col = torch.empty(max(pairs, 1), dtype=torch.int32).pin_memory().numpy()
    # the first calls with host points build this shape's launch plan and CUDA graph: warm-up
    e2e_ms = []
    e2e_warm = max(3, args.warmup)
    for k in range(max(3, args.steps // 2) + e2e_warm):
        flush(k)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.all_pairs(host_pts, r, T, r)
        row_ptr, col = res.download((host_rp, host_col))
        t1 = time.perf_counter()
        res.release()
        if k >= e2e_warm:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_value = pairs / (np.mean(e2e_ms) / 1e3)
    h2d = pts.nbytes + T.nbytes
    d2h = row_ptr.nbytes + col.nbytes

    # roofline of the dominant phase (per-phase device events over the timed region)
    mean_phase = {p: float(np.mean([ph[p] for ph in phases])) for p in phases[0]}
    pb = phase_bytes(n, d, m, key_bytes, passes, pts.dtype.itemsize, pairs)
    dom = max(pb, key=lambda p: mean_phase[p])
    peak, peak_kind = measured_peaks()
    achieved = pb[dom] / (mean_phase[dom] * 1e-6) / 1e9
    traffic = ncu_traffic(n, dtype_name, dom, sort_cfg)
    kernels = {"sort": "one k_sort_pass per radix pass (look-back), upsweep + scan + downsweep "
                       "per pass, or one k_sort_coop launch (autotuned variant)",
               "pairs": "k_pairs_warp + k_pairs_medium + k_large_setup + k_pairs_large"}[dom]
    roofline = {"bound": "hbm", "kernel": dom, "kernels": kernels, "achieved": round(achieved, 1),
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes": pb[dom], "launch_us": round(mean_phase[dom], 2),
                "bytes_model": "pairs: N (key + index) + N d S gather + 8 per pair (survey "
                               "per-grid model); sort: per radix pass read + write of the N "
                               "(key, index) elements"}
    return {
        "value": round(job_throughput(pairs, args.steps, ws, total_ms), 1),
        "ms_per_step": round(ms_per_step, 4), "total_ms": total_ms,
        "builds_per_s": round(args.steps * ws / (total_ms / 1e3), 2),
        "pairs_per_build": pairs, "exact_pairs": exact_pairs,
        "recall": round(pairs / exact_pairs, 5) if exact_pairs else 1.0,
        "p50_ms": round(float(np.percentile(step_ms, 50)), 4),
        "p99_ms": round(float(np.percentile(step_ms, 99)), 4),
        "wall_s_timed_region": round(wall_s, 3),
        "phase_us": {p: round(v, 2) for p, v in mean_phase.items()},
        "phase_bytes_model": info["phase_bytes"],
        "sort": sort_cfg, "enumeration": info["enumeration"], "roofline": roofline,
        "e2e": {"value": round(e2e_value, 1), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(float(np.mean(e2e_ms)), 4)},
        "clocks": clk, "gpu_launches": launches * args.steps,
    }


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1409_8112_gb300 import rtg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pts, T, r = workload()
    # torch and the library share one stream: inputs made by torch need no cross-stream wait
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = rtg.Context(local, stream=stream.cuda_stream)
    flush = L2Flush()
    rec = measure_build(ctx, stream, flush, args, pts, T, r, WORKLOAD.get("dtype", "fp64"), ws,
                        rank, clocks=ClockSampler(local))
    line = {
        "metric": METRIC, "value": rec["value"], "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic", "config": WORKLOAD,
    }
    for k in ("builds_per_s", "pairs_per_build", "exact_pairs", "recall", "p50_ms", "p99_ms",
              "wall_s_timed_region", "phase_us", "sort", "enumeration", "roofline", "e2e",
              "clocks", "gpu_launches"):
        line[k] = rec[k]
    line["phase_note"] = ("device phases from CUDA events on the library's stream, in a second "
                          "pass of the same steps (phase events add about 30 us a build, so the "
                          "timed steps run without them)")
    if args.config3 and WORKLOAD["n"] == 100000:
        # the 1,000,000-point FP32 build, measured in the same run with the same protocol
        set_workload(1000000, "fp32")
        p3, T3, r3 = workload()
        set_workload(100000, "fp64")
        c3 = measure_build(ctx, stream, flush, args, p3, T3, r3, "fp32", ws, rank,
                           clocks=ClockSampler(local))
        line["config3"] = {
            "workload": "rtg_all_pairs n=1000000 d=6 fp32 uniform[0,1]^6 r=2lnn-degree m=8 c=r "
                        "seed0",
            "metric": METRIC, "unit": "pairs/s", "dtype": "f32+f64", "steps": args.steps,
            **{k: c3[k] for k in ("value", "ms_per_step", "builds_per_s", "pairs_per_build",
                                  "exact_pairs", "recall", "p50_ms", "p99_ms", "phase_us",
                                  "sort", "enumeration", "roofline", "e2e", "clocks",
                                  "gpu_launches")},
        }
        line["gpu_launches"] += c3["gpu_launches"]
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pts, T, r, budget_s=args.cpu_seconds)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def cpu_baseline(pts, T, r, budget_s=12.0):
    """The oracle as it stands on whole builds of the same workload: on every host core
    (grids in parallel, then the merge by row ranges; ``value``) and on one core
    (``single_core``), each for about half of the budget."""
    import oracle
    cores = os.cpu_count() or 1

    def timed(fn, budget):
        times, pairs = [], 0
        t_start = time.perf_counter()
        while True:
            t0 = time.perf_counter()
            pairs = fn()
            times.append(time.perf_counter() - t0)
            if time.perf_counter() - t_start > budget or len(times) >= 20:
                break
        return pairs, times

    pa, ta = timed(lambda: oracle.rtg_threads(pts, r, T, r, cores).nnz, budget_s / 2)
    p1, t1 = timed(lambda: oracle.rtg(pts, r, T, r).csr.nnz, budget_s / 2)
    wl = f"n={pts.shape[0]}, d={pts.shape[1]}, m={len(T)}"
    return {"value": round(pa / float(np.median(ta)), 1), "unit": "pairs/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{len(ta)} complete build(s) of the bench workload ({wl}) on {cores} host "
                      f"threads, median {np.median(ta):.3f} s each",
            "single_core": {"value": round(p1 / float(np.median(t1)), 1), "cores": 1,
                            "sample": f"{len(t1)} complete build(s), median "
                                      f"{np.median(t1):.3f} s each"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    pts, T, r = workload()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.rtg_threads(pts, r, T, r, cores)
    times, pairs = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pairs = oracle.rtg_threads(pts, r, T, r, cores).nnz
        times.append(time.perf_counter() - t0)
    total = float(np.sum(times))
    value = pairs * args.steps / total
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "pairs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": WORKLOAD, "impl": "reference",
        "cpu_baseline": {"value": round(value, 1), "unit": "pairs/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{args.steps} complete builds of the bench workload on "
                                   f"{cores} host threads"},
        "e2e": {"value": round(value, 1), "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batch_workload(count=512, seed0=1000):
    """512 roadmaps: n log-uniform in [1e3, 2e5], d uniform in {3, 6, 9}, FP32 uniform
    points, r for expected degree 2 ln n, m = 6, seed 1000 + i (transforms c = r)."""
    from paper_1409_8112_gb300 import gen
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(np.floor(np.exp(rng.uniform(np.log(1e3), np.log(2e5)))))
        d = int(rng.choice([3, 6, 9]))
        pts = gen.points_uniform(seed0 + i, n, d, np.float32)
        r = gen.radius_for_degree(n, d)
        T = gen.transforms(seed0 + i, d, 6, r)
        out.append((pts, r, T, r))
    return out


def run_batch(args):
    """Batched form vs one build per roadmap, same 512 roadmaps, points resident on device."""
    import torch
    from paper_1409_8112_gb300 import rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    work = batch_workload()
    dev = [(torch.from_numpy(p).cuda(), r, T, c) for p, r, T, c in work]
    flush = L2Flush()
    for _ in range(args.warmup):
        res, offs = ctx.batch_all_pairs(dev, m=6)
        res.release()
    times, pairs = [], 0
    for k in range(args.steps):
        flush(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, offs = ctx.batch_all_pairs(dev, m=6, timing=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        pairs = res.nnz
        st = res.stats
        res.release()
    # one build per roadmap, every shape seen twice first (key width read back, sort variant
    # chosen, launch sequence captured) so that both forms are timed warm
    for _ in range(2):
        for p, r, T, c in dev:
            ctx.all_pairs(p, r, T, c).release()
    single_ms, single_pairs = [], 0
    for k in range(max(1, args.steps // 5)):
        flush(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tot = 0
        for p, r, T, c in dev:
            res = ctx.all_pairs(p, r, T, c)
            tot += res.nnz
            res.release()
        e1.record(stream)
        e1.synchronize()
        single_ms.append(e0.elapsed_time(e1))
        single_pairs = tot
    assert single_pairs == pairs, (single_pairs, pairs)
    ms = float(np.mean(times))
    sms = float(np.mean(single_ms))
    line = {
        "metric": METRIC, "value": round(pairs / (ms / 1e3), 1), "unit": "pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "batch of 512 roadmaps, n log-uniform [1e3,2e5], d in {3,6,9}, "
                               "fp32 uniform, r=2lnn-degree, m=6, seeds 1000+i",
                   "points": int(sum(len(w[0]) for w in work)), "l2": L2_NOTE},
        "builds_per_s": round(512 / (ms / 1e3), 1), "pairs_per_step": pairs,
        "one_build_per_roadmap": {"ms_per_512": round(sms, 3),
                                  "pairs_per_s": round(single_pairs / (sms / 1e3), 1),
                                  "builds_per_s": round(512 / (sms / 1e3), 1)},
        "speedup_vs_one_build_per_roadmap": round(sms / ms, 3),
        "phase_us": {k2: round(v, 1) for k2, v in st["phase_us"].items()},
        "key_bits": st["key_bits"], "sort_passes": st["sort_passes"], "sort": st["sort"],
        "enumeration": st["enumeration"],
        "gpu_launches": st["launches"] * args.steps,
    }
    ctx.close()
    print(json.dumps(line), flush=True)


def serve_shapes(count, rate, nmax, seed=7):
    """(arrival time, n, d) of every request of the serving trace, without its points."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(np.floor(np.exp(rng.uniform(np.log(1e3), np.log(nmax)))))
        d = int(rng.integers(2, 13))
        out.append((t, n, d))
    return out


def serve_request(i, n, d, seed=7):
    """Points, r and transforms of request i of the serving trace."""
    from paper_1409_8112_gb300 import gen
    pts = gen.points_mixture(seed * 100000 + i, n, d, k=8, sigma=0.05, dtype=np.float32)
    r = gen.radius_for_degree(n, d)
    T = gen.transforms(seed * 100000 + i, d, 8, r)
    return pts, r, T


def serve_trace(count, rate, nmax, seed=7):
    """Poisson arrivals; n log-uniform in [1e3, nmax]; d uniform in {2..12}; points from a
    mixture of 8 Gaussians (sigma 0.05, means in [0.1,0.9]^d) clipped to [0,1]^d, FP32;
    r for expected degree 2 ln n under uniform density; m = 8."""
    return [(t, *serve_request(i, n, d, seed))
            for i, (t, n, d) in enumerate(serve_shapes(count, rate, nmax, seed))]


def serve_run(ctx, trace, arrivals):
    """Submits the trace to the request server (at its arrival times, or all at once) while a
    client thread claims each result as soon as it is done (polling the outstanding tickets),
    so that no finished result holds memory.  Returns the served records and the makespan."""
    import queue
    import threading
    from paper_1409_8112_gb300 import rtg
    submitted = queue.Queue()
    rec = {"lat": [], "pairs": 0, "rejected": 0, "served": [], "slack": [], "corrected": 0}
    failure = []

    def claim():
        outstanding, left = {}, len(trace)
        while left:
            while True:
                try:
                    k, tk = submitted.get_nowait()
                except queue.Empty:
                    break
                outstanding[k] = tk
            done = 0
            for k in list(outstanding):
                try:
                    res = ctx.poll(outstanding[k], m=8)
                except rtg.RTGError as e:
                    del outstanding[k]
                    left -= 1
                    done += 1
                    if e.status == rtg.RTG_E_BUDGET:
                        rec["rejected"] += 1
                        continue
                    failure.append(e)
                    return
                if res is None:
                    continue
                del outstanding[k]
                left -= 1
                done += 1
                st = res.stats
                rec["corrected"] += st["attempts"] > 1
                rec["lat"].append(st["phase_us"]["total"] / 1e3)
                rec["pairs"] += res.nnz
                rec["served"].append(k)
                if st["mem_estimate"] > 0:
                    rec["slack"].append(st["mem_peak"] / st["mem_estimate"])
                res.release()
            if not done:
                time.sleep(0.0005)

    claimer = threading.Thread(target=claim)
    start = time.perf_counter()
    claimer.start()
    for k, (t0, pts, r, T) in enumerate(trace):
        if arrivals:
            now = time.perf_counter() - start
            if t0 > now:
                time.sleep(t0 - now)
        submitted.put((k, ctx.submit(pts, r, T, r)))
    claimer.join()
    if failure:
        raise failure[0]
    rec["makespan"] = time.perf_counter() - start
    return rec


def run_serve(args):
    """The request server on a Poisson trace (continuous batching over lanes, budget
    admission): latency at that load; then the same requests submitted at once (the server's
    capacity), and the same trace one build per request through rtg_all_pairs (no batching,
    no overlap).  Every build is exact, so each request has the same pair set (the same
    recall) in every form, and pairs/s compare directly."""
    import torch
    from paper_1409_8112_gb300 import rtg
    torch.cuda.set_device(0)
    budget = 64 << 30
    trace = serve_trace(args.requests, args.rate, args.nmax)
    warm = serve_trace(4, args.rate, args.nmax, seed=99)

    def server():
        # a fresh server (its lanes warmed with a few other requests), so that every request
        # of the trace is a shape it has not built before, as in a live stream
        c = rtg.Context(0, mem_budget_bytes=budget)
        for t0, pts, r, T in warm:
            c.wait(c.submit(pts, r, T, r), m=8).release()
        return c

    ctx = server()
    poisson = serve_run(ctx, trace, arrivals=True)
    ctx.close()
    ctx = server()
    burst = serve_run(ctx, trace, arrivals=False)
    # the same trace one request at a time, each a plain synchronous build (host points in),
    # the requests the budget refuses included (they fail there too)
    plain_ctx = rtg.Context(0, mem_budget_bytes=budget)
    for _, pts, r, T in warm:
        plain_ctx.all_pairs(pts, r, T, r).release()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_pairs, plain_refused, plain_corrected = 0, 0, 0
    for _, pts, r, T in trace:
        try:
            res = plain_ctx.all_pairs(pts, r, T, r)
        except rtg.RTGError as e:
            if e.status == rtg.RTG_E_BUDGET:
                plain_refused += 1
                continue
            raise
        plain_pairs += res.nnz
        plain_corrected += res.stats["attempts"] > 1
        res.release()
    plain_s = time.perf_counter() - t0
    plain_ctx.close()
    lat, slack = poisson["lat"], poisson["slack"]
    line = {
        "metric": METRIC, "value": round(poisson["pairs"] / poisson["makespan"], 1),
        "unit": "pairs/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"serving: Poisson {args.rate}/s, {args.requests} requests, n "
                               f"log-uniform [1e3,{args.nmax}], d in 2..12, 8-Gaussian mixture "
                               "sigma 0.05 fp32, r=2lnn-degree (uniform), m=8, budget 64 GiB"},
        "served": len(lat), "rejected_budget": poisson["rejected"],
        "p50_ms": round(float(np.percentile(lat, 50)), 3) if lat else None,
        "p99_ms": round(float(np.percentile(lat, 99)), 3) if lat else None,
        "builds_per_s": round(len(lat) / poisson["makespan"], 2),
        "makespan_s": round(poisson["makespan"], 3), "pairs": poisson["pairs"],
        "served_corrected": poisson["corrected"],
        "capacity": {
            "pairs_per_s": round(burst["pairs"] / burst["makespan"], 1),
            "pairs": burst["pairs"], "served": len(burst["lat"]),
            "rejected_budget": burst["rejected"],
            "builds_per_s": round(len(burst["lat"]) / burst["makespan"], 2),
            "seconds": round(burst["makespan"], 3), "corrected": burst["corrected"],
            "note": "the same requests submitted at once (no arrival times): the server "
                    "saturated"},
        "one_build_per_request": {
            "pairs_per_s": round(plain_pairs / plain_s, 1), "pairs": plain_pairs,
            "refused_budget": plain_refused,
            "builds_per_s": round((len(trace) - plain_refused) / plain_s, 2),
            "seconds": round(plain_s, 3), "corrected": plain_corrected,
            "note": "the whole trace back to back (no arrival times), one synchronous "
                    "rtg_all_pairs each, host points in"},
        "served_vs_one_by_one": round((burst["pairs"] / burst["makespan"]) /
                                      (plain_pairs / plain_s), 3),
        "comparison_note": "capacity (all requests at once) over one build per request, "
                           "pairs/s; every build is exact, so recall is equal",
        "corrected_note": "builds that had to correct a launch assumption (a pair buffer "
                          "sized for fewer pairs: a second enumeration writes the columns)",
        "admission_slack": {
            "peak_over_estimate_median": round(float(np.median(slack)), 3) if slack else None,
            "peak_over_estimate_max": round(float(np.max(slack)), 3) if slack else None,
            "note": "device bytes a batch needed (the workspace its build asked for and its "
                    "block CSR) over the batch's admission estimate"},
    }
    ctx.close()
    print(json.dumps(line), flush=True)


def run_clustered(args):
    """Clustered point sets (8 Gaussians, sigma 0.05, clipped to [0,1]^d; the serving
    workload's points) with r for expected degree 2 ln n under uniform density, m = 8, c = r,
    FP32: dense cells of thousands of points.  Each is built with the CUDA-core tiles and with
    the tensor-core tiles (FP16, BF16) for its cells of more than 256 points."""
    import torch
    from paper_1409_8112_gb300 import gen, rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()
    out = {}
    for n, d in ((200000, 6), (50000, 9), (100000, 3)):
        pts = torch.from_numpy(gen.points_mixture(5, n, d, k=8, sigma=0.05,
                                                  dtype=np.float32)).cuda()
        r = gen.radius_for_degree(n, d)
        T = gen.transforms(5, d, 8, r)
        rec = {}
        for tensor in (None, "fp16", "bf16"):
            for _ in range(args.warmup):
                ctx.all_pairs(pts, r, T, r, tensor=tensor).release()
            ms, ph = [], []
            for k in range(args.steps):
                flush(k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = ctx.all_pairs(pts, r, T, r, tensor=tensor)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                pairs = res.nnz
                res.release()
            res = ctx.all_pairs(pts, r, T, r, tensor=tensor, timing=True)
            st = res.stats
            res.release()
            rec[tensor or "cuda_cores"] = {
                "ms": round(float(np.mean(ms)), 3), "pairs": pairs,
                "pairs_per_s": round(pairs / (np.mean(ms) / 1e3), 1),
                "max_cell": st["max_cell"], "large_cells": st["large_cells"],
                "phase_ms": {p: round(v / 1e3, 3) for p, v in st["phase_us"].items()}}
        out[f"n{n}_d{d}"] = rec
    head = out["n200000_d6"]["cuda_cores"]
    line = {
        "metric": METRIC, "value": head["pairs_per_s"], "unit": "pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"],
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "clustered: 8 Gaussians sigma 0.05 fp32, r=2lnn-degree (uniform), "
                               "m=8, c=r, seed 5; n=200000 d=6 (headline), 50000 d=9, "
                               "100000 d=3", "l2": L2_NOTE},
        "builds": out,
    }
    ctx.close()
    print(json.dumps(line), flush=True)


def run_table2(args):
    """Shift-only RTG with the paper's Table II parameters (Sec. IV-A): d = 6, m = 20 grids,
    c = 1.35 r, r from Eq. 2, n uniform points in [0,1]^6 (FP64, seed 0).  Reported pairs/s
    at the recall Table II guarantees (>= 98%), beside the exact set on the same device
    (brute force, CUDA cores and FP16 tensor-core tiles, recall 1) and the rotated
    m = 8, c = r build of the headline workload (same points, its own radius)."""
    import torch
    from paper_1409_8112_gb300 import gen, rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()
    n, d, m, ct = args.n, 6, 20, 1.35
    r = gen.radius_fmt(n, d)
    pts = torch.from_numpy(gen.points_uniform(0, n, d)).cuda()
    T = gen.transforms(0, d, m, ct * r, flags=gen.SHIFT_ONLY)

    def timed(fn, reps, warm):
        for _ in range(warm):
            fn().release()
        ms, res = [], None
        for k in range(reps):
            flush(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if k + 1 < reps:
                res.release()
        return float(np.mean(ms)), res

    ms, res = timed(lambda: ctx.all_pairs(pts, r, T, ct * r, timing=True), args.steps, args.warmup)
    pairs, st = res.nnz, res.stats
    res.release()
    ex_ms, ex = timed(lambda: ctx.brute_force(pts, r, count_only=True), 3, 1)
    exact = ex.nnz
    ex.release()
    tc_ms, tc = timed(lambda: ctx.brute_force(pts, r, count_only=True, tensor="fp16"), 3, 1)
    assert tc.nnz == exact
    tc.release()
    line = {
        "metric": METRIC, "value": round(pairs / (ms / 1e3), 1), "unit": "pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"Table II shift-only RTG: n={n} uniform [0,1]^6 fp64, r from "
                               f"Eq. 2 ({r:.6f}), m={m}, c={ct} r, seed 0", "l2": L2_NOTE},
        "recall": round(pairs / exact, 5), "pairs_per_build": pairs, "exact_pairs": exact,
        "phase_us": {k: round(v, 1) for k, v in st["phase_us"].items()},
        "sort": dict(st["sort"], key_bits=st["key_bits"], passes=st["sort_passes"]),
        "exact_set_same_device": {
            "brute_force_cuda_cores_ms": round(ex_ms, 3),
            "brute_force_tensor_fp16_ms": round(tc_ms, 3),
            "pairs_per_s_cuda_cores": round(exact / (ex_ms / 1e3), 1),
            "pairs_per_s_tensor_fp16": round(exact / (tc_ms / 1e3), 1)},
        "speedup_vs_exact_tensor": round(tc_ms / ms, 2),
        "gpu_launches": st["launches"] * args.steps,
    }
    ctx.close()
    print(json.dumps(line), flush=True)


def run_params(args):
    """Grid parameters for a target recall (Sec. III-A): rtg_tune_params picks (c, m) for 98%
    recall on n uniform points in [0,1]^6 (FP64, seed 0, r from Eq. 2), shift-only and rotated;
    each choice is then built and timed like the headline, beside Table II's shift-only
    setting (m = 20, c = 1.35 r)."""
    import torch
    from paper_1409_8112_gb300 import gen, rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()
    n, d, target = args.n, 6, 0.98
    r = gen.radius_fmt(n, d)
    pts = torch.from_numpy(gen.points_uniform(0, n, d)).cuda()
    exact = ctx.brute_force(pts, r, count_only=True)
    n_exact = exact.nnz
    exact.release()

    def timed(T, c):
        for _ in range(args.warmup):
            ctx.all_pairs(pts, r, T, c).release()
        ms, pairs = [], 0
        for k in range(args.steps):
            flush(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = ctx.all_pairs(pts, r, T, c)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            pairs = res.nnz
            res.release()
        t = float(np.mean(ms))
        return {"ms_per_build": round(t, 4), "recall_full": round(pairs / n_exact, 5),
                "pairs_per_s": round(pairs / (t / 1e3), 1)}

    out = {}
    for name, shift in (("shift_only", True), ("rotated", False)):
        t0 = time.perf_counter()
        ch = ctx.tune_params(pts, r, target, seed=0, shift_only=shift)
        tune_s = time.perf_counter() - t0
        flags = gen.SHIFT_ONLY if shift else 0
        T = gen.transforms(0, d, ch["m"], ch["cell_side"], flags)
        out[name] = dict({"m": ch["m"], "c_over_r": ch["c_factor"],
                          "recall_sample": round(ch["recall"], 5), "tuning_s": round(tune_s, 3)},
                         **timed(T, ch["cell_side"]))
    T2 = gen.transforms(0, d, 20, 1.35 * r, gen.SHIFT_ONLY)
    out["table2_shift_only_m20_c1.35"] = timed(T2, 1.35 * r)
    best = min(("shift_only", "rotated"), key=lambda k: out[k]["ms_per_build"])
    line = {"metric": METRIC, "value": out[best]["pairs_per_s"], "unit": "pairs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out[best]["ms_per_build"], "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"tuned grids for recall >= {target}: n={n} uniform [0,1]^6 "
                                   f"fp64, r from Eq. 2 ({r:.6f}), seed 0", "l2": L2_NOTE},
            "exact_pairs": n_exact, "choices": out, "best": best}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_bitset(args):
    """Bit-matrix dedupe (Sec. III-B's flattened bit array) against the first-grid rule on the
    batched form: 512 small roadmaps, n log-uniform in [1e3, 16384], d in {3, 6, 9}, FP32
    uniform, r for degree 2 ln n, m = 6 and m = 20; same output, both timed warm."""
    import torch
    from paper_1409_8112_gb300 import gen, rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()
    rng = np.random.default_rng(11)
    ns = gen.log_uniform_int(rng, 1000, 16384, 512)
    ds = rng.choice([3, 6, 9], 512)
    out = {}
    for m in (6, 20):
        work = []
        for i, (n, d) in enumerate(zip(ns, ds)):
            r = gen.radius_for_degree(int(n), int(d))
            p = torch.from_numpy(gen.points_uniform(2000 + i, int(n), int(d), np.float32)).cuda()
            work.append((p, r, gen.transforms(2000 + i, int(d), m, r), r))
        res = {}
        for name, bits in (("first_grid", False), ("bitset", True)):
            for _ in range(args.warmup):
                ctx.batch_all_pairs(work, m=m, bitset=bits)[0].release()
            ms, pairs = [], 0
            for k in range(args.steps):
                flush(k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r_, _ = ctx.batch_all_pairs(work, m=m, bitset=bits)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                pairs = r_.nnz
                r_.release()
            t = float(np.mean(ms))
            res[name] = {"ms_per_batch": round(t, 3), "pairs": pairs,
                         "pairs_per_s": round(pairs / (t / 1e3), 1)}
        assert res["bitset"]["pairs"] == res["first_grid"]["pairs"]
        res["bitset_speedup"] = round(res["first_grid"]["ms_per_batch"] /
                                      res["bitset"]["ms_per_batch"], 3)
        out[f"m{m}"] = res
    line = {"metric": METRIC, "value": out["m6"]["bitset"]["pairs_per_s"], "unit": "pairs/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["m6"]["bitset"]["ms_per_batch"], "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch of 512 small roadmaps, n log-uniform [1e3,16384], d in "
                                   "{3,6,9}, fp32 uniform, r=2lnn-degree, m=6 and m=20",
                       "points": int(ns.sum()), "l2": L2_NOTE},
            "results": out}
    ctx.close()
    print(json.dumps(line), flush=True)


def run_query(args):
    """Multiple r-NN queries (Sec. II): the headline workload built once with every pair stored
    twice (symmetric CSR), then the neighbour lists of a random 10% of the points (host index
    list, repeats allowed) read back as a CSR, per step."""
    import torch
    from paper_1409_8112_gb300 import rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()
    pts, T, r = workload()
    n = len(pts)
    dev = torch.from_numpy(pts).cuda()
    g = ctx.all_pairs(dev, r, T, r, symmetric=True)
    q = np.random.default_rng(3).integers(0, n, n // 10).astype(np.int32)
    for _ in range(args.warmup):
        ctx.query_neighbors(g, q).release()
    ms, nnz = [], 0
    for k in range(args.steps):
        flush(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ctx.query_neighbors(g, q)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        nnz = res.nnz
        res.release()
    t = float(np.mean(ms))
    line = {"metric": METRIC, "value": round(nnz / (t / 1e3), 1), "unit": "neighbours/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t, 4),
            "higher_is_better": True, "dtype": "i32", "data": "synthetic",
            "config": {"workload": f"multiple r-NN queries: {len(q)} random indices into the "
                                   f"symmetric CSR of {WORKLOAD['workload']}", "l2": L2_NOTE},
            "queries": len(q), "neighbours_per_step": nnz,
            "queries_per_s": round(len(q) / (t / 1e3), 1), "graph_nnz": g.nnz}
    g.release()
    ctx.close()
    print(json.dumps(line), flush=True)


def run_points_query(args):
    """r-NN queries of new points from the stored grids (Sec. V): an index of the headline
    workload's m = 8 grids built once, then 100,000 new points uniform in [0,1]^6 (seed 9,
    host FP64) queried per step, their answers read back as a CSR; with the oracle's time on
    a 2,000-query sample of the same queries beside it."""
    import torch
    from paper_1409_8112_gb300 import rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()
    pts, T, r = workload()
    d = pts.shape[1]
    dev = torch.from_numpy(pts).cuda()
    t0 = time.perf_counter()
    ix = ctx.index(dev, r, T, r)
    build_s = time.perf_counter() - t0
    qs = np.random.default_rng(9).random((100000, d)).astype(pts.dtype)
    qdev = torch.from_numpy(qs).cuda()
    for _ in range(args.warmup):
        ix.query(qdev).release()
    ms, nnz = [], 0
    for k in range(args.steps):
        flush(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ix.query(qdev)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        nnz = res.nnz
        res.release()
    t = float(np.mean(ms))
    line = {"metric": METRIC, "value": round(len(qs) / (t / 1e3), 1), "unit": "queries/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t, 4),
            "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"r-NN queries of {len(qs)} new points uniform in [0,1]^6 "
                                   f"(seed 9) against the stored grids of {WORKLOAD['workload']}",
                       "l2": L2_NOTE},
            "answers_per_step": nnz, "answers_per_s": round(nnz / (t / 1e3), 1),
            "index_build_s": round(build_s, 4)}
    if not args.no_cpu_baseline:
        import oracle
        sample = qs[:2000]
        t0 = time.perf_counter()
        oracle.rtg_query(pts, r, T, r, sample)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": round(len(sample) / cpu_s, 1), "unit": "queries/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"{len(sample)} of the same queries against the same "
                                          f"points and grids, {cpu_s:.2f} s (grids rebuilt "
                                          f"per call)"}
    ix.close()
    ctx.close()
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Precision workload: n = 1e6 points of U[0,1]^6 stored FP32, r for degree 2 ln n, m = 8
    (RTG build), and the exact all-pairs set of a 200,000-point sample (first 200k points of a
    separate seeded draw, r for that n) on CUDA cores and on FP16 / BF16 tensor-core tiles."""
    import torch
    from paper_1409_8112_gb300 import gen, rtg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = rtg.Context(0, stream=stream.cuda_stream)
    flush = L2Flush()

    def timed(fn, reps):
        out, ms = None, []
        for k in range(reps):
            flush(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            if k + 1 < reps:
                out.release()
        return out, float(np.median(ms))

    n, d, m = 1000000, 6, 8
    r = gen.radius_for_degree(n, d)
    pts = torch.from_numpy(gen.points_uniform(0, n, d, np.float32)).cuda()
    T = gen.transforms(0, d, m, r)
    for _ in range(args.warmup):
        ctx.all_pairs(pts, r, T, r).release()
    build, build_ms = timed(lambda: ctx.all_pairs(pts, r, T, r, timing=True), args.steps)
    bst = build.stats
    nb = 200000
    rb = gen.radius_for_degree(nb, d)
    sample = torch.from_numpy(gen.points_uniform(1, nb, d, np.float32)).cuda()
    out = {}
    for name, tensor in (("cuda_cores_fp32", None), ("tensor_fp16", "fp16"),
                         ("tensor_bf16", "bf16")):
        ctx.brute_force(sample, rb, count_only=True, tensor=tensor).release()
        res, ms = timed(lambda: ctx.brute_force(sample, rb, count_only=True, tensor=tensor),
                        max(2, args.steps // 3))
        st = res.stats
        out[name] = {"ms": round(ms, 3), "pairs": res.nnz,
                     "pair_tests_per_s": round(nb * (nb - 1) / 2 / (ms / 1e3), 1),
                     "fp64_band_rechecks": st["dist_rechecks"],
                     "band": st["band"], "max_abs_err_d2": st["max_abs_err_d2"]}
        res.release()
    line = {
        "metric": METRIC, "value": round(build.nnz / (build_ms / 1e3), 1), "unit": "pairs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(build_ms, 3),
        "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "precision: n=1e6 U[0,1]^6 fp32, r=2lnn-degree, m=8; brute force "
                               "on a 200k sample", "l2": L2_NOTE},
        "rtg_pairs": build.nnz, "rtg_phase_us": {k: round(v, 1) for k, v in bst["phase_us"].items()},
        "rtg_key_bits": bst["key_bits"], "rtg_sort_passes": bst["sort_passes"],
        "brute_force_200k": out, "r_sample": rb, "r2_sample": rb * rb,
    }
    ctx.close()
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config3", dest="config3", action="store_false",
                    help="leave out the 1,000,000-point FP32 sub-record of the default line")
    ap.add_argument("--workload", default="build",
                    choices=["build", "batch", "serve", "precision", "table2", "query",
                             "points_query", "params", "bitset", "clustered"],
                    help="build: the headline single-roadmap workload; batch: 512 roadmaps "
                         "batched vs one by one; serve: a Poisson request trace")
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--nmax", type=int, default=500000)
    ap.add_argument("--n", type=int, default=100000,
                    help="points of the single-roadmap workload (headline: 100000)")
    ap.add_argument("--dtype", default="fp64", choices=["fp64", "fp32"],
                    help="coordinate type of the single-roadmap workload (headline: fp64)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    set_workload(args.n, args.dtype)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "table2":
        run_table2(args)
    elif args.workload == "query":
        run_query(args)
    elif args.workload == "points_query":
        run_points_query(args)
    elif args.workload == "params":
        run_params(args)
    elif args.workload == "bitset":
        run_bitset(args)
    elif args.workload == "clustered":
        run_clustered(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
