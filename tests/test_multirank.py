"""The multi-GPU benchmark's only cross-rank logic, on CPU: each rank solves its
own batch (no data-path collective) and the job time is the slowest rank's.
Two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(10.0 + 5.0 * rank)
    # the whole-job value is all ranks' units over the slowest rank's time
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        assert out[0] == 15.0 and out[1] == 15.0


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
