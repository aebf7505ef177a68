"""Replica timing aggregation across two ranks on CPU (gloo): the N > 1 path of the bench."""
import os

import pytest

from paper_2403_01596_gb300 import replicas


def _worker(rank, world_size, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world_size),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        r, lr, ws = replicas.world()
        replicas.barrier()
        slowest = replicas.max_over_ranks(1.5 + rank)  # rank 1 is the slower replica
        q.put((r, lr, ws, slowest, replicas.job_throughput(100.0, ws, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 0, 2), (1, 1, 2)]
    assert all(r[3] == 2.5 for r in res)           # both ranks see the slowest time
    assert all(r[4] == pytest.approx(80.0) for r in res)  # 2 x 100 units / 2.5 s


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.world() == (0, 0, 1)
    assert replicas.max_over_ranks(3.0) == 3.0
    with pytest.raises(ValueError):
        replicas.job_throughput(1.0, 1, 0.0)
