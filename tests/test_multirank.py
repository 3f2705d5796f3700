"""The N > 1 host logic of bench.py on two gloo ranks (CPU): replicas register
different pairs, the job time is the slowest rank's and the products add up;
the oracle reference arm prints on rank 0 only."""

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, n = bench.combine_ranks(1.0 + rank, 20 * (rank + 1), world, "cpu")
    out[rank] = (t, n, bench.rank_seed(1808, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_combination_over_gloo():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (t0, n0, s0), (t1, n1, s1) = out[0], out[1]
    assert t0 == t1 == 2.0            # slowest rank
    assert n0 == n1 == 60.0           # 20 + 40 products
    assert s0 != s1                   # each replica registers its own pair


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"workload": "3d_64_ellipsoids", "warmup": 3, "steps": 1, "gpus": 2})()
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
