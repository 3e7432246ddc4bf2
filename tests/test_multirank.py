"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2):
ranks get identical sections and their own target frames, and the reported
time is the max over ranks."""

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
    import torch
    import torch.distributed as dist

    import bench
    from paper_2506_02741_gb300 import synthetic as syn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    K = syn.scaled_intrinsics(48, 36)
    Kw, keys, section, targets, starts = bench.make_workload(rank, 2, K)
    mx = bench.reduce_max(10.0 + rank, world, torch.device("cpu"))
    out[rank] = (float(np.sum(section.depth)), float(np.sum(targets.depth)),
                 np.asarray(starts[0]).tolist(), mx)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0]                      # same section on every rank
    assert r0[1] != r1[1]                      # each rank tracks its own frames
    assert r0[2] != r1[2]
    assert r0[3] == r1[3] == 11.0              # max over ranks
