"""The multi-GPU form of bench.py is "replicas only": each rank runs its own
chain (its own seed) with no data-path collective, and rank 0 reports the
units of all ranks over the slowest rank's time. This checks that host
logic with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [400.0, 500.0][rank]
    rate, max_ms = bench.whole_job_rate(1000, local_ms, world, device="cpu")
    out[rank] = (bench.replica_seed(rank), rate, max_ms)
    dist.destroy_process_group()


def test_two_replicas_report_whole_job_rate():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    seeds = [out[r][0] for r in range(world)]
    assert len(set(seeds)) == world           # independent chains
    for r in range(world):
        assert out[r][2] == 500.0              # slowest rank's time
        assert out[r][1] == pytest.approx(2 * 1000 / 0.5)
