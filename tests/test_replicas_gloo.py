"""The replica plumbing of the benchmark (barrier, slowest-rank time,
whole-job rate) with two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1507_04891_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    r, w, lr = replicas.env()
    assert (r, w, lr) == (rank, world, rank)
    replicas.init(w, backend="gloo")
    replicas.barrier(w)
    t = 1.0 + rank            # rank 1 is the slow one
    tmax = replicas.max_over_ranks(t, w)
    out[rank] = (tmax, replicas.whole_job_rate(1000.0, tmax, w))
    replicas.finish(w)


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 1000.0)


def test_single_rank_needs_no_process_group():
    assert replicas.max_over_ranks(3.5, 1) == 3.5
    assert replicas.whole_job_rate(10.0, 2.0, 1) == 5.0
