"""Multi-rank decomposition on CPU ranks (gloo, world size 2), with the FP64 oracle standing in
for each rank's local operator: row-sharded R^dagger N^-1 with one all-reduce equals the
single-process result, channel sharding needs no exchange, and the timing reduction takes the
slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2406_09144_gb300.shard import RowSharded, channel_shard, max_over_ranks, shard_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleOp:
    def __init__(self, uvw, freqs, weights, nx, ny, pix):
        self.uvw, self.freqs, self.w = uvw, freqs, weights
        self.nx, self.ny, self.pix = nx, ny, pix

    def degrid(self, sky):
        import oracle
        return oracle.degrid(sky, self.uvw, self.freqs, self.pix, self.pix)

    def grid(self, vis):
        import oracle
        return torch.as_tensor(oracle.grid(vis, self.uvw, self.freqs, self.pix, self.pix, self.nx,
                                           self.ny, weights=self.w, nsky=1))


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2406_09144_gb300 import synth
    obs = synth.random_observation(90, 2, 12, 12, 2e-2, seed=5, wmax_cycles=1.5)
    vis = synth.complex_gaussian((obs.nrow, obs.nchan), seed=6)
    sky = synth.random_skies(1, 12, 12, seed=7)
    op = RowSharded(lambda u, f, w: OracleOp(u, f, w, 12, 12, obs.pixsize), obs.uvw, obs.freqs,
                    obs.weights, world, rank)
    dirty = op.grid(vis[op.start:op.stop]).numpy()
    local_vis = op.degrid(sky)
    t = max_over_ranks(1.0 + rank, world)
    out[rank] = (dirty, (op.start, op.stop), local_vis, t, channel_shard(8, world, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_row_sharded_gridding_equals_single_process():
    import oracle
    from paper_2406_09144_gb300 import synth
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn",
                       join=True)
    obs = synth.random_observation(90, 2, 12, 12, 2e-2, seed=5, wmax_cycles=1.5)
    vis = synth.complex_gaussian((obs.nrow, obs.nchan), seed=6)
    sky = synth.random_skies(1, 12, 12, seed=7)
    ref = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 12, 12,
                      weights=obs.weights, nsky=1)
    refv = oracle.degrid(sky, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize)
    for r in range(world):
        dirty, (a, b), lv, t, ch = out[r]
        assert np.allclose(dirty, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.allclose(lv, refv[a:b], rtol=1e-12, atol=1e-12)
        assert t == 2.0  # slowest rank
    assert out[0][1] == (0, 45) and out[1][1] == (45, 90)
    assert out[0][4] == (0, 4) and out[1][4] == (4, 8)


@pytest.mark.parametrize("n,world", [(10, 3), (7, 7), (3, 4), (0, 2)])
def test_shard_range_covers_everything_once(n, world):
    seen = []
    for r in range(world):
        a, b = shard_range(n, world, r)
        assert 0 <= a <= b <= n
        seen.extend(range(a, b))
    assert seen == list(range(n))


def _channel_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2406_09144_gb300 import synth
    from paper_2406_09144_gb300.shard import channel_slice
    obs = synth.random_observation(80, 4, 10, 10, 2e-2, seed=9, wmax_cycles=1.0,
                                   per_channel_sky=True)
    vis = synth.complex_gaussian((obs.nrow, obs.nchan), seed=10)
    c0, c1 = channel_shard(obs.nchan, world, rank)
    mine = channel_slice(obs, c0, c1)
    # each rank images its own channels from its own data: no collective on the data path
    dirty = oracle.grid(vis[:, c0:c1], mine.uvw, mine.freqs, mine.pixsize, mine.pixsize, 10, 10,
                        weights=mine.weights, nsky=c1 - c0)
    nvis = torch.tensor([float(mine.nvis)], dtype=torch.float64)
    dist.all_reduce(nvis)  # bench-side bookkeeping only: the job's visibility count
    out[rank] = (dirty, (c0, c1), float(nvis.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_channel_sharded_imaging_equals_single_process():
    """The benchmark's multi-GPU split of per-channel skies: ranks take disjoint channel ranges
    (shard.channel_slice), image them independently, and together give the single-process
    per-channel result; the visibility counts add up to the whole job's."""
    import oracle
    from paper_2406_09144_gb300 import synth
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_channel_worker, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn", join=True)
    obs = synth.random_observation(80, 4, 10, 10, 2e-2, seed=9, wmax_cycles=1.0,
                                   per_channel_sky=True)
    vis = synth.complex_gaussian((obs.nrow, obs.nchan), seed=10)
    ref = oracle.grid(vis, obs.uvw, obs.freqs, obs.pixsize, obs.pixsize, 10, 10,
                      weights=obs.weights, nsky=4)
    got = np.concatenate([out[r][0] for r in range(world)])
    assert [out[r][1] for r in range(world)] == [(0, 2), (2, 4)]
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert all(out[r][2] == obs.nvis for r in range(world))
