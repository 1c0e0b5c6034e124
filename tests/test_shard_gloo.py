"""Coloring sharding over ranks, on CPU with the gloo backend (world size 2 and 3).

Each rank counts its own contiguous range of seeds; the maps gathered from the
ranks must be the maps of all seeds counted in one process, and the estimate
from them the single-process estimate (Section 2.1: colorings are independent
iterations).  The per-rank counting here is the oracle's: the multi-rank host
logic is what is under test.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import sgcgen
from paper_1903_04395_gb300 import shard


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_total, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rp, ci = sgcgen.er(400, 1600, 3)
        parent = sgcgen.pruefer_tree(5, 11)
        seeds = shard.rank_seeds(100, n_total, rank, world)
        local = [oracle.count(rp, ci, parent, oracle.colors(int(s), len(rp) - 1, 5)).maps for s in seeds]
        full = shard.gather_maps(local, n_total)
        slowest = shard.max_over_ranks(float(rank + 1))
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([full, [slowest]]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_total", [(2, 7), (3, 10), (2, 1)])
def test_sharded_maps_equal_single_process(tmp_path, world, n_total):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, free_port(), n_total, str(tmp_path)), nprocs=world, join=True)
    rp, ci = sgcgen.er(400, 1600, 3)
    parent = sgcgen.pruefer_tree(5, 11)
    want = np.array([oracle.count(rp, ci, parent, oracle.colors(100 + i, len(rp) - 1, 5)).maps
                     for i in range(n_total)], dtype=np.float64)
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npy")
        assert np.array_equal(got[:-1], want), (r, got, want)
        assert got[-1] == world  # the slowest rank's value
    ref = oracle.estimate(rp, ci, parent, [100 + i for i in range(n_total)])
    # the estimate over every rank's maps, computed by the C library (no GPU needed)
    import paper_1903_04395_gb300 as sgc
    sgc.build()
    assert shard.estimate_from_maps(want, sgc.Template(parent)) == pytest.approx(ref.mean, rel=1e-12)


def test_shard_ranges_partition_the_seeds():
    for n_total in (0, 1, 5, 64, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shard.shard_range(n_total, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n_total
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(4, 2, 2)
