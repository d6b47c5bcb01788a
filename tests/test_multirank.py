"""The multi-rank (replicas) path of the benchmark on CPU: two gloo ranks.

The hot path shards by SNP blocks with no exchange, so N GPUs run N replicas; the only
cross-rank step is the benchmark's aggregation (slowest rank's time, units of all
ranks). That logic runs here with world_size 2 on the gloo backend.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
        el = bench.max_over_ranks(local_ms, world, "cpu")
        rate = bench.job_rate(16384 * 3, world, el / 1e3)
        # the reference arm runs on rank 0 only; other ranks leave without work
        ref = bench.run_reference(bench.parse_args_for_test([]), rank, world) if rank else None
        out[rank] = (el, rate, ref)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        el, rate, ref = out[r]
        assert el == pytest.approx(150.0)                   # slowest rank's time
        assert rate == pytest.approx(2 * 16384 * 3 / 0.150)  # units of all ranks
    assert out[1][2] is None
