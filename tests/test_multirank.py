"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own replicas; the job's
time is the slowest rank's, its work the sum over ranks, and the MFPT pools every replica."""
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, ev, fl = bench.combine_ranks(dist, "cpu", 100.0 + 50.0 * rank, 1000.0 * (rank + 1),
                                    np.array([rank + 0.5, rank + 0.25]))
    q.put((rank, t, ev, fl.tolist(), bench.rank_seeds(rank, 9)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, ev, fl, _ in out:
        assert t == 150.0                         # the slowest rank's time
        assert ev == 3000.0                       # work summed over ranks
        assert fl == [0.5, 0.25, 1.5, 1.25]       # every replica of every rank, rank order
    assert not set(out[0][4]) & set(out[1][4])    # disjoint seeds: independent replicas


def test_single_rank_passthrough():
    import bench
    t, ev, fl = bench.combine_ranks(None, "cpu", 12.5, 7.0, [1.0, 2.0])
    assert (t, ev) == (12.5, 7.0) and fl.tolist() == [1.0, 2.0]
