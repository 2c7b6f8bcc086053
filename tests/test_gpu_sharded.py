"""The sharded operator's default path on the GPU: library plans on CUDA tensors with the NCCL
collectives, in a one-rank process group (this pool gives one GPU per run; the two-rank logic
is covered on CPU by test_sharded_gloo.py).  With one rank it must equal the plain plan (grid
to rounding: summation order within a bucket differs between separately built plans)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_sharded_operator_one_rank_nccl():
    from paper_2010_10122_gb300 import _build
    _build.build()
    import torch.distributed as dist
    import paper_2010_10122_gb300 as wg
    from paper_2010_10122_gb300 import synthetic as S
    from paper_2010_10122_gb300.sharded import ShardedOperator
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        obs = S.random_uvw_observation(800, 4, 96, 64, 15.0, seed=71)
        op = ShardedOperator(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x,
                             obs.pixsize_y, 1e-10, "f64")
        plan = wg.Plan(obs.uvw, obs.freq, obs.npix_x, obs.npix_y, obs.pixsize_x, obs.pixsize_y,
                       1e-10, "f64")
        img = torch.from_numpy(S.gaussian_image(obs.npix_x, obs.npix_y, seed=1)).cuda()
        d = torch.from_numpy(S.complex_normal((obs.nrows, obs.nchan), seed=2)).cuda()
        assert op.rows == (0, obs.nrows)
        assert torch.equal(op.degrid(img.clone()), plan.degrid(img))
        # two separately built plans: the order inside a bucket comes from the bin-sort's
        # atomics, so gridding agrees to rounding
        a, b = op.grid(d), plan.grid(d)
        assert ((a - b).norm() / b.norm()).item() <= 1e-12
    finally:
        dist.destroy_process_group()
