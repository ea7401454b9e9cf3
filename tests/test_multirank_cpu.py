"""Host logic of the N>1 bench path on two gloo ranks (CPU): each rank simulates its own freshly
seeded batch (weak scaling, no data-path collective); only the timing is reduced (max over
ranks) and the body counts add up."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2607_06337_b300 import costs
from paper_2607_06337_b300 import inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    f = I.make_forest(I.BATCH, n_worlds=8, worlds=range(8), sweep=rank)  # the bench seeds rank r with sweep r
    bodies = torch.tensor([costs.body_count(f)], dtype=torch.float64)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)  # a rank's timed milliseconds
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(bodies, op=dist.ReduceOp.SUM)
    out[rank] = (float(t.item()), float(bodies.item()), int(f.body_off[-1]), float(f.k.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_host_logic():
    ws = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    t0, b0, nb0, k0 = out[0]
    t1, b1, nb1, k1 = out[1]
    assert t0 == t1 == 2.0                     # max over ranks
    assert b0 == b1                            # every rank sees the total
    f0 = I.make_forest(I.BATCH, n_worlds=8, worlds=range(8), sweep=0)
    f1 = I.make_forest(I.BATCH, n_worlds=8, worlds=range(8), sweep=1)
    assert b0 == costs.body_count(f0) + costs.body_count(f1)
    assert k0 != k1                            # the ranks hold different trees
