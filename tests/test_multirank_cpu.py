"""The multi-rank path on CPU (gloo, world size 2): disjoint realization ranges per rank,
max-over-ranks timing, and sharded results equal to the unsharded ones (the oracle stands in
for the GPU: a chain's trajectory depends only on its own seed / realization / stream)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys

    import torch
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 3
    rid0 = bench.shard_rid0(rank, n)
    t = bench.reduce_max_ms(10.0 + rank, world, device="cpu")
    energies = []
    for rid in range(rid0, rid0 + n):
        c = oracle.Chain(3, 4, 2, rid, 1)
        c.sweeps(20, oracle.quantize(3, np.zeros(c.b_top + 1)))
        energies.append(c.E)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rid0, energies))
    dist.barrier()
    out[rank] = (t, gathered)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    for r in range(world):
        t, gathered = out[r]
        assert t == 11.0                                  # the slowest rank's time
        assert [g[0] for g in gathered] == [0, 3]          # disjoint ranges
    # sharded energies equal the unsharded run of realizations 0..5
    import oracle
    want = []
    for rid in range(6):
        c = oracle.Chain(3, 4, 2, rid, 1)
        c.sweeps(20, oracle.quantize(3, np.zeros(c.b_top + 1)))
        want.append(c.E)
    got = out[0][1][0][1] + out[0][1][1][1]
    assert got == want
