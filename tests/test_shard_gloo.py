"""The N > 1 path on CPU: two gloo ranks take disjoint shards covering every solve, and the
step time is the maximum over ranks (no collective touches the solves' data)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO"])
import torch.distributed as dist
from paper_2603_29975_gb300 import shard
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + os.environ["PORT"], rank=rank, world_size=world)
atoms = list(shard.atom_range(rank, world, 64))
work = [(27 + (7 * i) % 143) ** 3 for i in range(50)]          # n^3 of uneven LIZ sizes
mine = shard.balance(work, world)[rank]
every = [None] * world
dist.all_gather_object(every, {"atoms": atoms, "mine": mine})
tmax = shard.max_over_ranks(1.5 + rank)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({"rank": rank, "every": every, "tmax": tmax}))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_shard_and_reduce():
    pytest.importorskip("torch.distributed")
    port = str(_free_port())
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", PORT=port, REPO=ROOT,
                   MASTER_ADDR="127.0.0.1", CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["tmax"] == 2.5
        a0, a1 = o["every"][0]["atoms"], o["every"][1]["atoms"]
        assert a0 == list(range(64)) and a1 == list(range(64, 128))
        m0, m1 = o["every"][0]["mine"], o["every"][1]["mine"]
        assert sorted(m0 + m1) == list(range(50)) and not set(m0) & set(m1)
    work = [(27 + (7 * i) % 143) ** 3 for i in range(50)]
    l0 = sum(work[i] for i in outs[0]["every"][0]["mine"])
    l1 = sum(work[i] for i in outs[0]["every"][1]["mine"])
    assert abs(l0 - l1) <= max(work)                   # greedy balance within one solve


def test_balance_and_ranges_single_process():
    from paper_2603_29975_gb300 import shard
    assert list(shard.atom_range(1, 4, 3)) == [3, 4, 5]
    with pytest.raises(ValueError):
        shard.atom_range(4, 4, 3)
    parts = shard.balance([5, 1, 4, 2, 3], 2)
    assert parts == [[0, 1, 3], [2, 4]]                # 5, 4, 3, 2, 1 in turn: loads 8 and 7
    assert shard.balance([], 3) == [[], [], []]
    assert shard.max_over_ranks(3.25) == 3.25          # no process group
