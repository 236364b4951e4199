"""The benchmark's multi-rank aggregation, on CPU with the gloo backend.

With N ranks the benchmark runs one independent lattice per rank and reports
the slowest rank's time (and every rank's kernel launches).  Two CPU ranks
check that reduction; no GPU is involved.
"""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed, launches = bench.reduce_over_ranks(dist, 1.5 + rank, 100 * (rank + 1), "cpu")
    out[rank] = (elapsed, launches)
    dist.destroy_process_group()


def test_slowest_rank_and_total_launches():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert dict(out) == {0: (2.5, 300), 1: (2.5, 300)}
