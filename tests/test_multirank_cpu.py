"""The N > 1 launch of bench.py on CPU ranks (gloo, world size 2, 127.0.0.1):
every rank projects its own cloud (distinct seeds), the job time is the
maximum over ranks, the throughput counts every rank's points, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_setup(None)
        step, fwd = bench.max_over_ranks(local_ms[rank], "cpu")
        value = bench.job_throughput(w, 1000, step)
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "ref_sample": 10})()) if r != 0 else "rank0"
        out[rank] = (w, r, step, fwd, value, bench.rank_seeds(r), ref)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_points():
    port = _free_port()
    local_ms = {0: [10.0, 4.0], 1: [12.5, 3.0]}
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, local_ms, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        w, r, step, fwd, value, seeds, _ = res[rank]
        assert (w, r) == (2, rank)
        assert step == 12.5 and fwd == 4.0            # element-wise maximum over the ranks
        assert value == pytest.approx(2 * 1000 / 12.5e-3)
    assert res[0][5] != res[1][5]                     # each rank its own cloud and cotangent
    assert res[1][6] is None                          # the reference arm: rank 0 alone runs


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.0]) == [3.0, 1.0]
    assert bench.job_throughput(1, 2_000_000, 10.0) == pytest.approx(2e8)
