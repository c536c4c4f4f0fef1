"""Replica timing on two gloo ranks (CPU): barrier, max-over-ranks job time and
whole-job throughput, as bench.py uses them under torchrun."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1904_02471_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t_local = [0.5, 2.0][rank]
    t = replicas.job_time(dist, t_local)
    out[rank] = (t, replicas.whole_job_rate(100.0, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_time_is_the_max_and_rate_counts_all_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (2.0, 100.0)


def test_single_process():
    assert replicas.job_time(None, 1.5) == 1.5
    assert replicas.whole_job_rate(10.0, 1, 2.0) == 5.0
    with pytest.raises(ValueError):
        replicas.whole_job_rate(1.0, 1, 0.0)
