"""The multi-GPU path of the benchmark runs independent replicas (the update has no exchange step in this
build): every rank times its own copy of the workload and the job's rate is the units of all ranks over
the slowest rank's time. These CPU tests run that reduction over world_size-2 gloo process groups."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w = bench._dist()
        slowest = bench.max_over_ranks(times[rank], w)
        rate = bench.replica_rate(1000.0, slowest, w)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{r} {w} {slowest!r} {rate!r}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.5, 2.0), (3.0, 1.0)])
def test_replica_timing_takes_the_slowest_rank(tmp_path, times):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), list(times), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    rows = [open(tmp_path / f"rank{k}.txt").read().split() for k in range(world)]
    for k, (r, w, slowest, rate) in enumerate(rows):
        assert int(r) == k and int(w) == world
        assert float(slowest) == max(times)
        assert float(rate) == world * 1000.0 / max(times)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.replica_rate(10.0, 2.0, 1) == 5.0
