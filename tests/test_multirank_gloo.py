"""The replicas-over-ranks bookkeeping of bench.py with two gloo ranks on CPU: the job time
is the slowest rank's, the work the sum of the ranks' dofs, and every rank agrees."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, dofs = bench.combine_over_ranks(10.0 + 5.0 * rank, 1000 + rank, tdist, "cpu")
    out.put((rank, ms, dofs))
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 2001), (1, 15.0, 2001)]


def test_single_rank_passthrough():
    import bench
    assert bench.combine_over_ranks(3.5, 42) == (3.5, 42)
