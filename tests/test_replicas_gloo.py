"""Multi-rank host logic of the benchmark, on CPU with the gloo backend and
two ranks: every rank runs its own replica of the workload with distinct
seeds, the slowest rank sets the time, and the whole-job rate counts the units
of all ranks.  Runs contain no collective on the data path (the APO runs of
different replicas share nothing), so this is the whole N > 1 path."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch
import bench
world, rank, local = bench.replica_setup("gloo")
# a fake per-rank time: rank r took 1 + r seconds for 1000 units
t = bench.max_over_ranks(1.0 + rank, world)
bench.sync_ranks(world)
seeds = [bench.replica_seed(k, rank) for k in range(5)]
out = {{"world": world, "rank": rank, "t_max": t, "seeds": seeds,
        "rate": bench.aggregate_rate(world, 1000, t)}}
with open(os.path.join({tmp!r}, "rank%d.json" % rank), "w") as f:
    json.dump(out, f)
torch.distributed.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_max_and_distinct_seeds(tmp_path):
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        code = CHILD.format(root=ROOT, tmp=str(tmp_path))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT))
    for p in procs:
        assert p.wait(timeout=120) == 0
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    for r, d in enumerate(res):
        assert d["world"] == 2 and d["rank"] == r
        assert d["t_max"] == 2.0                       # the slowest rank's time on every rank
        assert d["rate"] == pytest.approx(2 * 1000 / 2.0)
    # replicas draw different random numbers: no seed is shared between ranks
    assert not set(res[0]["seeds"]) & set(res[1]["seeds"])


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.aggregate_rate(1, 100, 2.0) == 50.0
    assert len({bench.replica_seed(k, r) for k in range(10) for r in range(8)}) == 80
