"""The N > 1 path of bench.py on the CPU: two ranks in a gloo process group
(the bench uses NCCL, one rank per GPU), each with its own step time, as
`bench.py --gpus 2` under torchrun would have them.  The step time reported
is the slowest rank's, and the whole-job rate counts the work of every
replica over that time (weak scaling: each rank solves its own system)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT_DIR"])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
ms = bench.ranks_max(50.0 + 10.0 * rank, dist, "cpu")       # rank r took 50 + 10 r ms
rate = bench.replica_rate(1.0e12, ms / 1e3, world)           # 1e12 flop per rank
alone = bench.ranks_max(7.0)                                  # no process group: the value itself
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "world": world, "ms": ms, "rate": rate, "alone": alone}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_replica_rate():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT_DIR=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2
        assert o["ms"] == 60.0                      # the slower rank's time, on every rank
        assert o["rate"] == 2 * 1.0e12 / 0.060      # both replicas' work over that time
        assert o["alone"] == 7.0
