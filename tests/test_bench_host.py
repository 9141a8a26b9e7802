"""Host-side logic of bench.py without a GPU: the replica plumbing (barrier,
max over ranks) on two gloo ranks, and the reference arm's rank rule."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, argparse
sys.path.insert(0, sys.argv[1])
import bench
args = argparse.Namespace(impl="ours")
world, rank, local = bench.dist_setup(args, backend="gloo")
assert world == 2 and rank in (0, 1)
bench.barrier(world)
m = bench.max_over_ranks(world, float(10 * (rank + 1)), "cpu")
assert m == 20.0, m
# the slowest rank's time defines the job's time: value = all units / max time
ms = bench.max_over_ranks(world, [1.5, 2.5][rank], "cpu")
assert ms == 2.5
import torch.distributed as dist
dist.destroy_process_group()
print("rank", rank, "ok")
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_replica_plumbing_on_two_gloo_ranks():
    port = _free_port()
    procs = []
    for rank in (0, 1):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=120)[0] for p in procs]
    for p, o in zip(procs, outs):
        assert p.returncode == 0, o
    assert "rank 0 ok" in outs[0] and "rank 1 ok" in outs[1]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(impl="reference", steps=1, warmup=0, gpus=2))
    assert capsys.readouterr().out == ""
