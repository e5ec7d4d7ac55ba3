"""The benchmark's multi-rank plumbing on two gloo ranks (CPU): barrier, max-over-ranks timing and
distinct per-rank scans (weak scaling, replicas; the imaging path has no data-path collective)."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = bench.max_over_ranks(1.5 + rank, world, "cpu")
    rot = [bench.scan_rotation(b, rank) for b in range(bench.N_BUF)]
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, t, rot))


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
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
    assert [r[1] for r in res] == [2.5, 2.5]                 # both ranks report the slowest rank's time
    assert set(res[0][2]).isdisjoint(res[1][2])              # each rank images its own (rotated) scans
