"""Multi-GPU decomposition of the measurement operator (one process per GPU).

The operator splits two ways:
  * by channel (per-channel skies, nsky = nchan): every channel is an independent imaging problem
    (its own grid, w-planes and PSF), so ranks take disjoint channel ranges and exchange nothing;
  * by visibility rows (one sky for all channels, or more visibilities than one GPU holds):
    R (Eq. rime) needs the sky on every rank and produces each rank's own visibilities; R^dagger
    N^-1 (Eq. clean) is a sum over visibilities, so each rank grids its rows and one all-reduce
    (sum) of the nx * ny dirty image completes it. The image is far smaller than the grids, so
    this is the cheapest place to exchange.
The local operator is anything with degrid(sky) / grid(vis) (binding.Plan on a GPU); the
collective is torch.distributed (NCCL on GPUs, gloo on CPU ranks in the tests).
"""
from __future__ import annotations

from typing import Callable, Tuple

import numpy as np


def shard_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous, balanced split of n items over `world` ranks: [start, stop) of `rank`."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


class RowSharded:
    """R / R^dagger N^-1 over visibility rows split across ranks.

    make_local(uvw_rows, freqs, weights_rows) builds this rank's operator; rows [start, stop) of
    the observation are this rank's. grid() returns the full dirty image on every rank."""

    def __init__(self, make_local: Callable, uvw, freqs, weights, world: int, rank: int,
                 group=None):
        self.start, self.stop = shard_range(len(uvw), world, rank)
        w = None if weights is None else np.asarray(weights)[self.start:self.stop]
        self.local = make_local(np.asarray(uvw)[self.start:self.stop], freqs, w)
        self.group = group
        self.world = world

    def degrid(self, sky):
        """This rank's visibilities, rows [start, stop)."""
        return self.local.degrid(sky)

    def grid(self, vis_local):
        """Full R^dagger N^-1 V: local gridding, then one sum all-reduce of the image."""
        import torch
        import torch.distributed as dist
        d = self.local.grid(vis_local)
        t = d if isinstance(d, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(d))
        if self.world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t


def channel_shard(nchan: int, world: int, rank: int) -> Tuple[int, int]:
    """Channels [start, stop) imaged by `rank` when skies are per channel (no communication)."""
    return shard_range(nchan, world, rank)


def max_over_ranks(value: float, world: int, group=None) -> float:
    """Maximum of a per-rank timing over all ranks (the slowest rank defines the step time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def channel_slice(obs, start: int, stop: int):
    """The observation restricted to channels [start, stop): the rows and uvw stay, the
    frequencies, weights and noise levels keep only those channels (per-channel skies, so the
    slice is a complete imaging problem of its own)."""
    import dataclasses
    if not 0 <= start < stop <= len(obs.freqs):
        raise ValueError(f"channel range [{start}, {stop}) outside 0..{len(obs.freqs)}")
    return dataclasses.replace(obs, freqs=np.asarray(obs.freqs)[start:stop],
                               weights=np.ascontiguousarray(np.asarray(obs.weights)[:, start:stop]),
                               sigma=np.ascontiguousarray(np.asarray(obs.sigma)[:, start:stop]))
