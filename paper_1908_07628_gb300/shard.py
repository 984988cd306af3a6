"""Detector-beam sharding of the inelastic map across processes.

The map is a sum of |.|^2 over detector beams (the detector sum of Eq. SHn0 applied
to each probe), so G processes can each run `Context.inelastic_map` on one shard of
the EELS aperture (`Context.set_detector_shard(g, G)`: beams d with d mod G == g) and
add their FP64 maps.  Every process needs the full S_in; S_out and the contraction
split G ways.  The sum here runs in a fixed order (rank 0, 1, ..., G-1), so every
rank holds the same bits, and they equal `sum_maps` of the same maps on one host.
"""
from __future__ import annotations


def detector_shard(n_out: int, index: int, count: int) -> list:
    """Indices of the detector beams (aperture enumeration order) in shard `index`."""
    if count < 1 or not 0 <= index < count:
        raise ValueError("need 0 <= index < count")
    return list(range(index, n_out, count))


def sum_maps(maps):
    """FP64 sum of shard maps in list order (numpy arrays or torch tensors)."""
    out = maps[0].copy() if hasattr(maps[0], "copy") else maps[0].clone()
    for m in maps[1:]:
        out += m
    return out


def allreduce_map(local, group=None):
    """Sum a torch FP64 map over the ranks of `group` in rank order; returns the sum
    on every rank.  Uses all_gather (no reduction inside the collective), so the
    result does not depend on the backend's reduction order."""
    import torch
    import torch.distributed as dist
    if local.dtype != torch.float64:
        raise TypeError("the map is FP64")
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    return sum_maps(parts)
