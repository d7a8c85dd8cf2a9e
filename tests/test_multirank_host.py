"""The benchmark's N-replica aggregation with two gloo ranks on the CPU.

With N GPUs the benchmark runs N independent replicas (nothing on the data
path is exchanged). The whole-job figure is every rank's keys over the
slowest rank's step time, so each rank must see the maximum of the ranks'
times. Two processes on the gloo backend stand in for two GPUs.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(times[rank], w, "cpu")
        rate = bench.job_mkeys_per_s(1_000_000, w, ms)
        dist.barrier()
        out.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(6.5, 7.25), (9.0, 3.0)])
def test_two_ranks_agree_on_the_slowest_step(times):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    want_rate = 2 * 1_000_000 / (slowest / 1e3) / 1e6
    assert sorted(r[0] for r in results) == [0, 1]
    for rank, world, local, ms, rate in results:
        assert (world, local) == (2, rank)
        assert ms == slowest
        assert rate == pytest.approx(want_rate, rel=1e-12)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.5, 1, "cpu") == 4.5
    assert bench.job_mkeys_per_s(150_000_000, 1, 7.5) == pytest.approx(20_000.0)
