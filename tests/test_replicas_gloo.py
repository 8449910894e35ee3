"""Multi-rank host logic of the benchmark, run as two gloo ranks on CPU:
every rank gets its own seeded problem (replicas, weak scaling) and the
timed region is reduced by max over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ws_, rank_, local_ = bench.dist_env()
    mk = bench.make_markers("multidrop1024", seed_offset=rank_)
    t = bench.max_over_ranks(10.0 + rank_)
    out.put((rank_, ws_, float(mk.X[0]), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_timing():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, x0, t0), (r1, w1, x1, t1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert x0 != x1            # independent seeded problems per rank
    assert t0 == t1 == 11.0    # max over ranks


def test_single_process_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
