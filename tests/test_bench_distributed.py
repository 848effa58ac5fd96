"""The replicas path of bench.py on CPU: 2 gloo ranks, disjoint chain ranges, max-over-ranks timing."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, world)
    off = bench.replica_chain_offset(rank, 1024)
    v = bench.aggregate_throughput(1024 * 100 * 3, world, m)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, off, v))


def test_two_rank_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, o0, v0), (r1, m1, o1, v1) = res
    assert m0 == m1 == 150.0                  # both ranks see the slowest time
    assert (o0, o1) == (0, 1024)              # disjoint Philox chain words
    assert v0 == v1 == pytest.approx(2 * 1024 * 100 * 3 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.aggregate_throughput(10, 1, 1000.0) == 10.0
