"""The N > 1 launch of bench.py (replicas, one process per GPU) on CPU ranks over gloo: the
job's timed region is the slowest rank's, the whole-job throughput counts every rank's builds,
and the reference arm prints from rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
ws, rank, _ = bench.dist_env()
own = [12.5, 40.0][rank]                  # this rank's timed-region milliseconds
total = bench.max_over_ranks(own, ws, device="cpu")
value = bench.job_throughput(1000, 10, ws, total)
print(json.dumps({{"rank": rank, "total": total, "value": value}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, ws=2):
    port = _free_port()
    procs = []
    for rank in range(ws):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   WORLD_SIZE=str(ws), RANK=str(rank), LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_and_job_throughput():
    import json
    outs = _run_ranks(WORKER.format(root=ROOT))
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["total"] == 40.0               # the slower replica sets the job's time
        assert r["value"] == pytest.approx(1000 * 10 * 2 / 0.040)


def test_reference_arm_rank_nonzero_exits_quietly():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
