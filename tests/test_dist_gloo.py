"""Two CPU processes (gloo, world size 2) each sample a contiguous block of
chains with the FP64 oracle; their merged moments equal the single-process
run's, and every chain's final state equals its single-process state bit for
bit (the Metropolis stream depends only on the global chain index)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_22718_gb300 import dist as rdist
from paper_2604_22718_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, total, out_dir):
    import torch.distributed as dist
    from oracle import oracle as orc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    inst = inputs.workload("tiny_fp64")
    o = orc.Oracle(inst)
    chain0, count = rdist.shard(total, rank, world)
    spins = inputs.initial_spins(5, total, inst.n_spins)[chain0:chain0 + count].copy()
    mant, ex = o.init_chains(spins)
    trace, _ = o.mcmc(22719, spins, mant, ex, 0, 6, chain0=chain0)
    merged = rdist.merge_moments(trace)
    np.save(os.path.join(out_dir, f"spins{rank}.npy"), spins)
    if rank == 0:
        np.save(os.path.join(out_dir, "merged.npy"), np.array([merged["n"], merged["mean"], merged["var"]]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_blocks_cover_the_range():
    for total in (0, 1, 7, 64, 4097):
        for world in (1, 2, 3, 8):
            blocks = [rdist.shard(total, r, world) for r in range(world)]
            assert sum(c for _, c in blocks) == total
            pos = 0
            for c0, c in blocks:
                assert c0 == pos
                pos += c


def test_two_gloo_ranks_reproduce_one_process(tmp_path):
    from oracle import oracle as orc
    total, world = 21, 2
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, total, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    inst = inputs.workload("tiny_fp64")
    o = orc.Oracle(inst)
    spins = inputs.initial_spins(5, total, inst.n_spins)
    mant, ex = o.init_chains(spins)
    trace, _ = o.mcmc(22719, spins, mant, ex, 0, 6)
    got = np.concatenate([np.load(tmp_path / f"spins{r}.npy") for r in range(world)])
    assert np.array_equal(got, spins)
    n, mean, var = np.load(tmp_path / "merged.npy")
    assert n == trace.size
    assert mean == pytest.approx(trace.mean(), rel=1e-13)
    assert var == pytest.approx(trace.var(), rel=1e-10)
