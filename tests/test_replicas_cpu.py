"""The N > 1 path of bench.py on CPU: replicas aggregated over a gloo
process group of world size 2 (slowest rank's time, units of all ranks), and
the reference arm printing on rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 10 * (r + 1) units
        t, u = bench.replica_totals(dist, 1.0 + rank, 10.0 * (rank + 1))
        out[rank] = (t, u)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_totals_gloo_world2():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, u = res[rank]
        assert t == 2.0                 # the slowest replica
        assert u == 30.0                # units of both replicas


def test_replica_totals_single_process():
    import bench
    assert bench.replica_totals(None, 1.5, 7.0) == (1.5, 7.0)


def test_reference_arm_prints_on_rank0_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    args = SimpleNamespace(config=bench.WORKLOAD, warmup=3, steps=1, cpu_rows=8)
    with redirect_stdout(buf):
        assert bench.run_reference(args) is None
    assert buf.getvalue() == ""
