"""Multi-process (world size 2, gloo, CPU) checks of the history sharding of
the multi-GPU path: the int64 all-reduce is exact beyond 2^53; run_sharded
splits the history range, reduces the ranks' int64 tallies and converts the
sum once (with a stand-in engine whose tally is an integer function of the
histories it replayed); and ranks replaying disjoint ranges with the oracle
add up to one process replaying every history."""
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


class _FakeEngine:
    """Stands in for fdc.Engine on the CPU: the 'tally' of histories
    [h0, h0 + n) puts 2^40 + h units into voxel h mod nvox for each history h
    (large integers, so a float reduction would lose bits)."""

    def __init__(self, nvox):
        self.device = 0
        self.shape = (nvox,)
        self.calls = []

    def run_ex(self, spots, n, seed, history_offset=0, tally=None, **kw):
        self.calls.append((history_offset, n))
        t = torch.zeros(self.shape, dtype=torch.int64)
        for h in range(history_offset, history_offset + n):
            t[h % self.shape[0]] += (1 << 40) + h
        tally.copy_(t)

    def sync(self):
        return {}

    def dose_from_tally(self, tally, dose=None):
        return tally.to(torch.float64) * 0.5


def _expected_fake(nvox, h0, n):
    t = torch.zeros((nvox,), dtype=torch.int64)
    for h in range(h0, h0 + n):
        t[h % nvox] += (1 << 40) + h
    return t


def _worker_int64(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1011_2188_gb300.shard import all_reduce_tally, run_sharded
    # exactness beyond 2^53: float64 would round these sums
    big = torch.tensor([(1 << 62) - 1 - rank, (1 << 53) + 1, -(1 << 60) + 3 * rank], dtype=torch.int64)
    all_reduce_tally(big)
    eng = _FakeEngine(37)
    tally = torch.zeros((37,), dtype=torch.int64)
    t, d = run_sharded(eng, None, 1001, 5, rank, world, tally=tally, history_offset=20)
    if rank == 0:
        torch.save({"big": big, "tally": t, "dose": d, "calls": eng.calls}, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_int64_all_reduce_and_run_sharded_two_ranks(tmp_path):
    out = str(tmp_path / "r.pt")
    mp.start_processes(_worker_int64, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    r = torch.load(out)
    want = [((1 << 62) - 1) + ((1 << 62) - 2), 2 * ((1 << 53) + 1), -(1 << 61) + 3]
    want = [((w + (1 << 63)) % (1 << 64)) - (1 << 63) for w in want]  # int64 wrap-around of the first
    assert r["big"].tolist() == want
    assert r["calls"] == [(20, 500)]  # rank 0: histories [20, 520) of [20, 1021)
    exp = _expected_fake(37, 20, 1001)
    assert torch.equal(r["tally"], exp)
    assert torch.equal(r["dose"], exp.to(torch.float64) * 0.5)
