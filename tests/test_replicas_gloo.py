"""The multi-GPU path is replicas only: every rank runs an independent
population (its own run tag, hence its own Philox field streams), with no
data-path collective; the bench takes the slowest rank's time and the units
of all ranks. These checks run that host logic as two gloo ranks on the CPU,
with the oracle standing in for each rank's walkers."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

WORLD = 2
STEPS = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(s, steps):
    from oracle import afqmc as O
    orc = O.OracleRun(s)
    for _ in range(steps):
        orc.step()
    return np.concatenate([orc.weight, orc.logO.real, orc.logO.imag])


def _rank_main(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        import bench
        from synth import small_system
        # the bench's workload carries the rank as its run tag
        assert bench.workload("c1", rank).run_id == rank
        # slowest rank's time, on every rank
        t = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        assert t == 10.0 + 5.0 * (WORLD - 1)
        # this rank's replica: same system, its own run tag
        s = small_system(M=6, n_up=2, n_dn=2, n_chol=5, seed=3, n_walkers=8,
                         ortho_every=2, measure_every=3, pc_every=3).replace(run_id=rank)
        mine = torch.tensor(_replica(s, STEPS), dtype=torch.float64)
        parts = [torch.zeros_like(mine) for _ in range(WORLD)]
        dist.all_gather(parts, mine)
        if rank == 0:
            np.save(os.path.join(out_dir, "replicas.npy"), torch.stack(parts).numpy())
    finally:
        dist.destroy_process_group()


def test_replicas_are_independent_and_reproducible(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(port, str(tmp_path)), nprocs=WORLD, join=True)
    got = np.load(tmp_path / "replicas.npy")
    from synth import small_system
    for rank in range(WORLD):
        s = small_system(M=6, n_up=2, n_dn=2, n_chol=5, seed=3, n_walkers=8,
                         ortho_every=2, measure_every=3, pc_every=3).replace(run_id=rank)
        # each rank's population is what a single process with that tag computes
        np.testing.assert_array_equal(got[rank], _replica(s, STEPS))
    # different tags draw different fields: the replicas are not copies
    assert np.max(np.abs(got[0] - got[1])) > 1e-6


def test_whole_job_value_counts_every_rank():
    import bench
    # 1024 walkers x 20 steps x 10 blocks per rank, 2 ranks, slowest 100 ms
    v = bench.whole_job_value(1024 * 20 * 10, 2, 100.0)
    assert v == pytest.approx(2 * 1024 * 20 * 10 / 0.1)
