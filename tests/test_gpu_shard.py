"""Sharded run of the engine (GB300): two processes on the same GPU each
replay half of the history range through the C ABI, their int64 tallies are
summed with an all-reduce (gloo, staged through host memory; the kernels of
the two processes never wait on each other) and converted to dose once.  The
result equals one process replaying every history, bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_1011_2188_gb300 import synth

pytestmark = pytest.mark.gpu


def _inputs():
    db = synth.water_database(synth.database_energies(24), 100, seed=2, nuclear=True)
    ph = synth.thorax_phantom(seed=7, shape=(96, 96, 64))
    beam = synth.field_beam(60001, energy=150.0, width=8.0, height=8.0)
    return db, ph, beam


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    from paper_1011_2188_gb300 import fdc
    from paper_1011_2188_gb300.shard import run_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    db, ph, beam = _inputs()
    eng = fdc.Engine(0)
    eng.load_database(db)
    eng.load_phantom(ph)
    tally, dose = run_sharded(eng, beam, 60001, 4, rank, world, track_group=32)
    torch.cuda.synchronize()
    if rank == 0:
        np.savez(out_path, tally=tally.cpu().numpy(), dose=dose.cpu().numpy())
    eng.close()
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_add_up_to_one_run_bitwise(tmp_path):
    import torch
    import torch.multiprocessing as mp
    import __graft_entry__
    __graft_entry__.build()
    from paper_1011_2188_gb300 import fdc
    out = str(tmp_path / "sharded.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    got = np.load(out)
    db, ph, beam = _inputs()
    eng = fdc.Engine(0)
    eng.load_database(db)
    eng.load_phantom(ph)
    shape = ph.shape[::-1]
    tally = torch.zeros(shape, dtype=torch.int64, device="cuda:0")
    dose = torch.zeros(shape, dtype=torch.float64, device="cuda:0")
    eng.run_ex(beam, 0, 4, tally=tally, dose=dose, track_group=32)
    eng.sync()
    assert np.array_equal(got["tally"], tally.cpu().numpy())
    assert np.array_equal(got["dose"], dose.cpu().numpy())
    # the conversion of a caller-held tally is the run's own finalize
    d2 = eng.dose_from_tally(tally)
    assert torch.equal(d2, dose)
    eng.close()
