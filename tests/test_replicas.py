"""Multi-process host logic of bench.py (replicas only: every rank solves the
whole workload; no data-path collective).  Two gloo ranks on the CPU: the
timing reduction gives every rank the slowest rank's time, the whole-job value
counts every rank's units, and the rank environment is parsed as torchrun sets it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
    torch.distributed.barrier()
    out.put((rank, slowest, bench.job_value(1000, ws, slowest * 1e-3)))
    torch.distributed.destroy_process_group()


def test_two_rank_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]                       # both see the slowest rank
    assert all(abs(r[2] - 2000 / 0.015) < 1e-6 for r in res)         # units of both ranks / slowest time
