"""The multi-rank path of bench.py on CPU with gloo (world size 2): each
rank takes its own contiguous shard of the state stream (weak scaling, no
collective on the data path) and the reported time is the maximum over
ranks."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    n = 1000
    start, count = bench.shard(rank, n)
    T, p, Y = bench.make_inputs(rank, n)
    t = bench.max_over_ranks(float(rank + 1) * 10.0, dist, torch.device("cpu"))
    out[rank] = (start, count, float(T[0]), float(Y[0, -1]), t)
    dist.destroy_process_group()


def test_two_ranks_shard_and_max_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    (s0, c0, T0, y0, t0), (s1, c1, T1, y1, t1) = out[0], out[1]
    assert (s0, c0, s1, c1) == (0, 1000, 1000, 1000)          # disjoint, contiguous, covering
    assert t0 == t1 == 20.0                                   # every rank sees the slowest time
    import bench
    from paper_2411_02640_gb300 import synth
    m = synth.mechanism(bench.MECH)
    T, p, Y = synth.make_states(m.n_species, synth.STATE_SPECS[bench.MECH], 0, 2000)
    assert T0 == T[0] and T1 == T[1000] and y1 == Y[0, 1999]  # the shards are the global stream's
