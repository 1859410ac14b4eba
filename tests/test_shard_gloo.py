"""Multi-process (world size 2, gloo, CPU) check of the history sharding used
by the multi-GPU replica path: ranks replay disjoint history ranges with the
oracle, the per-rank energy grids are summed with an all-reduce, and the
result equals one process replaying every history."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1011_2188_gb300.shard import shard_range, weak_shard


def test_shard_range_partitions():
    for total in (0, 1, 7, 1000, 12345):
        for world in (1, 2, 3, 8):
            parts = [shard_range(total, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == total
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    assert weak_shard(100, 3) == (300, 400)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1011_2188_gb300 import synth
    from paper_1011_2188_gb300.shard import all_reduce_tally, shard_range
    db = synth.water_database([120.0], 50, seed=3)
    ph = synth.slab_phantom(n=24, voxel_cm=0.5)
    beam = synth.pencil_beam(3001, energy=120.0, sigma_cm=0.5)
    lo, hi = shard_range(3001, rank, world)
    r = oracle.run(db, ph, beam, seed=17, h_begin=lo, h_end=hi)
    t = torch.from_numpy(r.edep.copy())
    all_reduce_tally(t)
    n = torch.tensor([r.n_histories], dtype=torch.int64)
    all_reduce_tally(n)
    if rank == 0:
        np.save(out_path, t.numpy())
        assert int(n[0]) == 3001
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sum_equals_single_process(tmp_path):
    import oracle
    from paper_1011_2188_gb300 import synth
    oracle.build()
    out = str(tmp_path / "sum.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    db = synth.water_database([120.0], 50, seed=3)
    ph = synth.slab_phantom(n=24, voxel_cm=0.5)
    beam = synth.pencil_beam(3001, energy=120.0, sigma_cm=0.5)
    ref = oracle.run(db, ph, beam, seed=17).edep
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9)
