"""The multi-rank host path of bench.py on CPU: world_size-2 gloo ranks aggregate the
slowest rank's time and the summed work; the reference arm's non-zero ranks exit at once."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
ms, work = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), "cpu", world)
print(json.dumps({{"rank": rank, "ms": ms, "work": work}}))
dist.destroy_process_group()
"""


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_gloo_two_ranks_aggregate():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    import json
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        d = json.loads(o.strip().splitlines()[-1])
        assert d["ms"] == 150.0 and d["work"] == 3000.0


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--workload", "cantilever3d_64x32x32"], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    import json
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config",
              "cpu_baseline", "e2e"):
        assert k in d
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_batch_shard_covers_every_problem_once():
    import bench
    items = list(range(48))
    for world in (1, 2, 3, 4, 8):
        parts = [bench.shard(items, r, world) for r in range(world)]
        assert sorted(x for p in parts for x in p) == items
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
