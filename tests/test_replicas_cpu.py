"""The multi-rank path of the benchmark on CPU (gloo, world size 2).

On N GPUs every rank evaluates an independent replica of the workload; the
job's time is the slowest rank's and its throughput counts every rank's
pairs.  This checks the cross-rank reduction and the aggregate on two gloo
ranks, and that the reference arm leaves the work to rank 0.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
        slowest = bench.max_over_ranks(local_ms)
        value = bench.job_throughput(1_000_000, 10, world, slowest)
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})()) if rank == 1 else None
        out.put((rank, slowest, value, ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value, ref in results:
        assert slowest == 150.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(1_000_000 * 10 * 2 / 0.150)
        assert ref is None  # only rank 0 runs the reference arm
