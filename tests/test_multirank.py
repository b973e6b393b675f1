"""Host logic of the multi-process benchmark path, on CPU with gloo ranks.

Every rank runs one replica of the workload (independent sources: no
collective on the data path); the only cross-rank step is the MAX of the timed
region, and the reference arm runs on rank 0 alone."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, value = bench.job_seconds_per_unit([120.0, 180.0][rank], 3, world, "cpu")
        dist.barrier()
        ref = bench.run_reference(None, rank) if rank != 0 else "skipped"
        out.put((rank, ms, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value, ref in res:
        assert ms == 180.0                                # slowest rank's timed region
        assert value == pytest.approx(180.0 / 1e3 / (3 * world))   # steps x world units
    assert res[1][3] is None                              # reference arm: rank 1 does no work


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.job_seconds_per_unit(250.0, 5, 1)
    assert ms == 250.0 and value == pytest.approx(0.05)

