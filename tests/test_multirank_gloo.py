"""World-size-2 CPU test (gloo) of the multi-rank host logic of the batched
benchmark: every mesh of the sweep is solved by exactly one rank, loads are
balanced by longest-processing-time, and the step time is the maximum over
ranks."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2509_06347_b300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = synth.batch_cylinder_specs()
    sizes = [2 * s["n_theta"] * s["n_r"] * 16 for s in specs]
    mine = bench.lpt_partition(sizes, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)  # this rank's elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((gathered, float(t.item()), sizes))
    dist.destroy_process_group()


def test_two_ranks_partition_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, sizes = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    allm = sorted(gathered[0] + gathered[1])
    assert allm == list(range(len(sizes)))
    loads = [sum(sizes[i] for i in part) for part in gathered]
    assert max(loads) - min(loads) <= max(sizes)
    assert tmax == 2.0
