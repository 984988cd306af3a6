"""Detector-beam sharding: the host side on two gloo ranks (CPU, no GPU).

The map is a sum over detector beams of |.|^2 (Eq. SHn0 applied to each probe), so
the maps of disjoint detector shards add up to the full map.  Each rank computes
the FP64 oracle map of its shard (beams d with d mod 2 == rank, the rule the
library's EELS_OPT_SHARD_* options state) and the ranks add them with
`shard.allreduce_map`; the total must equal the full oracle map to rounding and be
bit-identical to the same sum taken in rank order on one host.
"""
import os

import numpy as np
import pytest

import specimen as sp
from oracle import linear as lin
from oracle import multislice as ms
from paper_1908_07628_gb300 import shard

WORLD = 2


def _workload():
    return sp.random_workload(n=32, n_z=3, f=1, cell=8.0, n_sites=4, w=6, seed=77,
                              alpha=0.012, beta=0.018, dz=1.5, scan_n=3)


def _rank_main(rank, store_path, out_dir):
    import torch
    import torch.distributed as dist
    store = dist.FileStore(store_path, WORLD)
    dist.init_process_group("gloo", store=store, rank=rank, world_size=WORLD)
    try:
        wl = _workload()
        n_out = ms.lattice_beams(wl.n, wl.cell, wl.lam, wl.f, wl.beta)[0].size
        mine = lin.linear_map(wl, detectors=np.array(shard.detector_shard(n_out, rank, WORLD)))
        total = shard.allreduce_map(torch.from_numpy(mine))
        np.save(os.path.join(out_dir, f"part{rank}.npy"), mine)
        np.save(os.path.join(out_dir, f"total{rank}.npy"), total.numpy())
    finally:
        dist.destroy_process_group()


def test_detector_shards_sum_to_the_full_map_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    tmp.spawn(_rank_main, args=(str(tmp_path / "store"), str(tmp_path)), nprocs=WORLD,
              join=True)
    parts = [np.load(tmp_path / f"part{r}.npy") for r in range(WORLD)]
    totals = [np.load(tmp_path / f"total{r}.npy") for r in range(WORLD)]
    for t in totals:   # same bits on every rank, equal to the rank-order host sum
        assert np.array_equal(t, shard.sum_maps(parts))
    full = lin.linear_map(_workload())
    assert full.max() > 0 and all(p.max() > 0 for p in parts)
    assert ms.relative_error(full, totals[0]) < 1e-12


def test_shard_indices_partition_the_aperture():
    for n_out, count in [(1, 1), (7, 3), (5, 8), (1321, 4)]:
        seen = sorted(d for g in range(count) for d in shard.detector_shard(n_out, g, count))
        assert seen == list(range(n_out))
    with pytest.raises(ValueError):
        shard.detector_shard(10, 2, 2)
