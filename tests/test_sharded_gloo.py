"""Visibility sharding over processes (Sec. 4.4: split the measurement set over nodes, broadcast
the image for degridding, sum the images after gridding), checked with world_size 2 on the gloo
backend (CPU, 127.0.0.1 rendezvous).  The per-rank operator here is the FP64 direct-sum oracle,
so the test pins the partitioning and the collectives: the ranks' visibilities put together and
the summed image must equal the oracle on the whole data set."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2010_10122_gb300 import synthetic as S
from paper_2010_10122_gb300.sharded import row_block

OBS = dict(nrows=301, nchan=3, npix_x=32, npix_y=48, fov_deg=15.0, seed=61)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OraclePlan:
    """The per-rank operator of the test: the direct sums of Eq. (rime) and its adjoint."""

    def __init__(self, uvw, freq, nx, ny, psx, psy, epsilon, precision):
        self.uvw, self.freq, self.nx, self.ny, self.psx, self.psy = uvw, freq, nx, ny, psx, psy

    def degrid(self, dirty):
        from oracle import direct
        return torch.from_numpy(direct.degrid(self.uvw, self.freq, dirty.numpy(), self.psx, self.psy))

    def grid(self, vis):
        from oracle import direct
        return torch.from_numpy(direct.grid(self.uvw, self.freq, vis.numpy(), self.nx, self.ny,
                                            self.psx, self.psy))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2010_10122_gb300.sharded import ShardedOperator
    obs = S.random_uvw_observation(**OBS)
    op = ShardedOperator(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                         1e-12, "f64", make_plan=OraclePlan)
    img = torch.from_numpy(S.gaussian_image(obs.npix_x, obs.npix_y, seed=1))
    if rank != 0:
        img.zero_()                      # only rank 0 holds the image; degrid broadcasts it
    vis = op.degrid(img)
    r0, r1 = op.rows
    d = torch.from_numpy(S.complex_normal((obs.nrows, obs.nchan), seed=2)[r0:r1])
    dirty = op.grid(d)
    q.put((rank, op.rows, vis.numpy(), dirty.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_row_blocks_cover_the_rows_evenly():
    for nrows, world in ((301, 2), (7, 3), (2, 4), (0, 2), (1000, 8)):
        blocks = [row_block(nrows, world, r) for r in range(world)]
        assert blocks[0][0] == 0 and blocks[-1][1] == nrows
        assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
        sizes = [b - a for a, b in blocks]
        assert max(sizes) - min(sizes) <= 1


def test_sharded_operator_two_ranks(oracle_lib):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    obs = S.random_uvw_observation(**OBS)
    I = S.gaussian_image(obs.npix_x, obs.npix_y, seed=1)
    d = S.complex_normal((obs.nrows, obs.nchan), seed=2)
    rv = oracle_lib.degrid(obs.uvw, obs.freq, I, obs.pixsize_x, obs.pixsize_y)
    ri = oracle_lib.grid(obs.uvw, obs.freq, d, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y)
    assert [x[1] for x in res] == [(0, 151), (151, 301)]
    vis = np.concatenate([x[2] for x in res])
    assert np.array_equal(vis, rv)                  # each visibility's sum is the same sum
    for x in res:                                   # every rank holds the summed image
        assert np.linalg.norm(x[3] - ri) <= 1e-13 * np.linalg.norm(ri)
