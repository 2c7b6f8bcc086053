"""The N > 1 benchmark path runs independent replicas; its only cross-rank steps are a barrier
and max / sum reductions of timings and counts.  Checked with world_size 2 on the gloo backend
(CPU, 127.0.0.1 rendezvous)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2010_10122_gb300 import replicas
    ws, r, lr = replicas.world()
    mx = replicas.max_over_ranks(10.0 + rank)
    sm = replicas.sum_over_ranks(1000 + rank)
    dist.barrier()
    q.put((r, ws, lr, mx, sm))
    dist.destroy_process_group()


def test_replica_reductions_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert all(x[3] == 11.0 and x[4] == 2001.0 for x in res)


def test_single_process_identity():
    from paper_2010_10122_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
