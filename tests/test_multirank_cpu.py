"""The benchmark's N > 1 path on CPU: two gloo ranks (world size 2).

With N GPUs every rank advances its own realization (weak scaling, no
collective on the data path); the only communication is the barrier around
the timed region and the max over ranks of its duration.  These tests run
that host logic (process-group set-up from the torchrun environment, the
barrier, the max reduction, the per-rank workload seeds) in two processes.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    bench.init_dist(w, "gloo")
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 + rank, w)
    wl = bench.rank_workload(rank, n=48)
    digest = float(np.sum(wl.eps * np.arange(wl.eps.size).reshape(wl.eps.shape) % 997))
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{m} {wl.seed} {digest} {wl.grid[0]}\n")
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    # both ranks see the max of the per-rank durations
    assert float(rows[0][0]) == float(rows[1][0]) == 11.0
    # each rank has its own realization: different noise seeds and disorder
    assert rows[0][1] != rows[1][1]
    assert rows[0][2] != rows[1][2]
    assert rows[0][3] == rows[1][3] == "48"


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)          # a no-op without a process group
