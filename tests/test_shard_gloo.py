"""Weak-scaling shard logic with two gloo ranks on the CPU.

Each rank runs its own trajectory counters (here with the oracle, standing in
for the device); the union gathered on rank 0 equals the run of all
trajectories in one process, and the job time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1412_2293_gb300 import inputs, shard

N, PER_RANK, E, SEED, X0 = 6, 3, 0.05, 1234, 5


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import circuits as ocirc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.trajectory_range(rank, PER_RANK)
        ops = inputs.qft_circuit(N)
        fids = ocirc.trajectory_fidelities(N, ops, X0, E, SEED, range(lo, hi))
        allf = shard.gather_to_rank0(fids, dist)
        tmax = shard.max_over_ranks(1.0 + rank, dist)
        if rank == 0:
            np.save(os.path.join(out_dir, "fids.npy"), allf)
            np.save(os.path.join(out_dir, "tmax.npy"), np.array([tmax]))
        else:
            assert allf is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_cover_the_single_process_run(tmp_path):
    from oracle import circuits as ocirc
    world = 2
    mp.start_processes(rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "fids.npy")
    want = ocirc.trajectory_fidelities(N, inputs.qft_circuit(N), X0, E, SEED, range(world * PER_RANK))
    np.testing.assert_array_equal(got, want)
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0


def test_shard_helpers_single_process():
    assert shard.trajectory_range(0, 4) == (0, 4)
    assert shard.trajectory_range(3, 4) == (12, 16)
    with pytest.raises(ValueError):
        shard.trajectory_range(-1, 4)
    assert shard.max_over_ranks(2.5) == 2.5
    np.testing.assert_array_equal(shard.gather_to_rank0(np.arange(3.0)), np.arange(3.0))
    assert shard.job_throughput(100.0, 4, 2.0) == 200.0
