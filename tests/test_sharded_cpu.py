"""Host logic of a grid split along z into slabs (CPU): the partition, the
point-to-point exchange of boundary planes between neighbouring ranks, and
the FP64 sum of the read-outs over the ranks, run as gloo ranks (world
sizes 2 and 3) with CPU tensors standing in for the device planes."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_0809_1547_gb300.sharded import slab_partition  # noqa: E402


@pytest.mark.parametrize("nz,parts,npml", [(48, 2, 8), (48, 3, 8), (320, 8, 8), (37, 3, 4),
                                           (19, 2, 8), (448, 4, 8), (40, 1, 8), (24, 5, 4)])
def test_partition_covers_the_grid_with_cuts_outside_the_cpml(nz, parts, npml):
    b = slab_partition(nz, parts, npml)
    assert len(b) == parts and b[0][0] == 0 and b[-1][1] == nz
    for (a0, a1), (c0, c1) in zip(b, b[1:]):
        assert a1 == c0                                  # contiguous, no overlap
    for z0, z1 in b:
        assert z1 > z0                                   # every slab owns a plane
    for _, c in b[:-1]:
        assert npml + 1 <= c <= nz - npml - 1            # ghosts c-1, c outside the z-CPML
    sizes = [z1 - z0 for z0, z1 in b]
    if parts > 1 and nz >= 4 * (npml + 1) * parts:       # room to balance: within one plane
        assert max(sizes) - min(sizes) <= 1


def test_partition_rejects_what_cannot_be_cut():
    assert slab_partition(18, 2, 8) == [(0, 9), (9, 18)]      # the one cut plane, 9
    with pytest.raises(ValueError):
        slab_partition(18, 3, 8)          # two cuts need two planes in [9, 9]
    with pytest.raises(ValueError):
        slab_partition(16, 2, 8)          # no plane in [9, 7]
    with pytest.raises(ValueError):
        slab_partition(10, 0, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_0809_1547_gb300.sharded import exchange_planes, reduce_readouts, slab_partition
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank's boundary planes, marked with (rank, side) in every element
    n = 1000
    send_lo = torch.full((n,), 10.0 * rank + 0.0)
    send_hi = torch.full((n,), 10.0 * rank + 1.0)
    recv_lo = torch.full((n,), -1.0)
    recv_hi = torch.full((n,), -1.0)
    for _ in range(3):                    # the exchange repeats every step
        exchange_planes(send_lo, send_hi, recv_lo, recv_hi, rank, world)
    # the read-outs: energy and six face energies of this rank's slab
    vals = np.array([1.0 + rank] + [rank * 1e-3 + q for q in range(6)], dtype=np.float64)
    tot = reduce_readouts(vals)
    bounds = slab_partition(48, world, 8)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(" ".join(str(v) for v in [float(recv_lo[0]), float(recv_lo.min()),
                                          float(recv_hi[0]), float(recv_hi.max())] + list(tot)
                         + [bounds[rank][0], bounds[rank][1]]) + "\n")
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_planes_and_sum_readouts(tmp_path, world):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    rows = [[float(v) for v in open(tmp_path / f"rank{r}.txt").read().split()] for r in range(world)]
    for r, row in enumerate(rows):
        lo0, lo_min, hi0, hi_max = row[:4]
        # from below: rank r-1's highest own plane; nothing on the first rank
        assert lo0 == lo_min == (10.0 * (r - 1) + 1.0 if r > 0 else -1.0)
        # from above: rank r+1's lowest own plane; nothing on the last rank
        assert hi0 == hi_max == (10.0 * (r + 1) + 0.0 if r < world - 1 else -1.0)
        tot = row[4:11]
        assert tot[0] == sum(1.0 + q for q in range(world))
        for q in range(6):
            assert tot[1 + q] == pytest.approx(sum(p * 1e-3 + q for p in range(world)), rel=1e-15, abs=0)
    # the ranks' slabs tile the grid
    spans = [(int(r[11]), int(r[12])) for r in rows]
    assert spans == slab_partition(48, world, 8)
