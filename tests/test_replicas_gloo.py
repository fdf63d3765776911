"""The replica (multi-rank) logic of the benchmark, run as two gloo ranks on CPU."""
import os
import socket

import pytest

from paper_0712_0813_gb300.replicas import aggregate_throughput, max_over_ranks, replica_seed


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_0712_0813_gb300 import replicas
    replicas.barrier(dist)
    t = replicas.max_over_ranks(1.5 + rank, dist)       # rank 1 is the slowest
    q.put((rank, t, replicas.replica_seed(1, rank)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]
    assert [o[2] for o in out] == [1, 2]          # each replica evolves its own lattice


def test_single_process_helpers():
    assert max_over_ranks(3.0) == 3.0
    assert aggregate_throughput(4, 1e9, 2.0) == 2e9
    assert replica_seed(7, 3) == 10
