"""Host-side logic of bench.py's multi-GPU launch (replicas, one rank per GPU),
run as two gloo ranks on the CPU: the job's time is the slowest rank's, the job's
throughput counts every rank's clusters, and the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, world)            # rank 1 is the slow one
    v = bench.replica_throughput(world, 1728, 3, t)
    dist.barrier()
    rc = bench.run_reference(None) if rank == 1 else None  # non-zero ranks exit without work
    dist.destroy_process_group()
    q.put((rank, t, v, rc))


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    assert all(o[2] == pytest.approx(2 * 1728 * 3 / 2.0) for o in out)
    assert out[1][3] == 0


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(1, 10, 2, 4.0) == 5.0
