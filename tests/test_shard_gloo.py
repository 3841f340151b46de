"""Multi-rank path on CPU: two gloo ranks run disjoint job ranges (here through
the oracle, standing in for one GPU each) and merge their FP64 accumulators;
the result equals the single-process run bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1411_3487_gb300 import shard

M, C, STEPS, DTAU = 16, 9, 20, 1.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _chain_sums(jobs):
    """Per-chain trajectory end state and observable sums, one row per job id."""
    m = O.Model(M, dtau=DTAU)
    R = np.stack([m.equilibrium_start(4, int(j)) for j in jobs])
    sums = np.zeros((len(jobs), 4))
    for s in range(STEPS):
        R = m.run_modes(R, 4, np.asarray(jobs), s, 1)
        for i in range(len(jobs)):
            o = m.observables(R[i])
            sums[i] += [o[0], o[1], o[2], 1.0]
    return R.reshape(len(jobs), -1), sums


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        jobs = list(shard.job_range(rank, world, C))
        R, sums = _chain_sums(jobs)
        allR = shard.gather_chains(R, C)
        total = shard.merge_sums(sums, C)
        np.save(os.path.join(out_dir, f"R{rank}.npy"), allR)
        np.save(os.path.join(out_dir, f"S{rank}.npy"), total)
    finally:
        dist.destroy_process_group()


def test_job_ranges_partition_the_chains():
    for n in (0, 1, 7, 4096):
        for w in (1, 2, 3, 8):
            got = [j for r in range(w) for j in shard.job_range(r, w, n, base=5)]
            assert got == list(range(5, 5 + n))
    with pytest.raises(ValueError):
        shard.job_range(2, 2, 10)


def test_two_gloo_ranks_merge_bit_exactly(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    R1, S1 = _chain_sums(list(range(C)))
    ref_sum = np.zeros(4)
    for row in S1:
        ref_sum += row
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"R{r}.npy"), R1)
        assert np.array_equal(np.load(tmp_path / f"S{r}.npy"), ref_sum)
