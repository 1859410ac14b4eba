"""The oracle is reentrant: runs over disjoint history ranges in parallel
threads (how the benchmark times it on every host core) add up to one
sequential run over the union of the ranges."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
from paper_1011_2188_gb300 import synth


def test_parallel_ranges_add_up_to_one_run():
    db = synth.water_database([150.0], 200, seed=1)
    ph = synth.slab_phantom()
    beam = synth.pencil_beam(2400, energy=150.0, sigma_cm=0.3)
    whole = oracle.run(db, ph, beam, seed=9, h_begin=0, h_end=2400)
    cuts = [0, 500, 1100, 1800, 2400]
    with ThreadPoolExecutor(4) as ex:
        parts = list(ex.map(lambda i: oracle.run(db, ph, beam, seed=9, h_begin=cuts[i], h_end=cuts[i + 1]),
                            range(4)))
    assert sum(p.n_histories for p in parts) == whole.n_histories == 2400
    assert sum(p.n_steps for p in parts) == whole.n_steps
    assert sum(p.n_segments for p in parts) == whole.n_segments
    np.testing.assert_allclose(sum(p.edep for p in parts), whole.edep, rtol=1e-12, atol=1e-9)
    assert abs(sum(p.escaped for p in parts) - whole.escaped) <= 1e-9 * max(1.0, whole.escaped)


def test_run_parallel_equals_one_run():
    db = synth.water_database([150.0], 200, seed=1, nuclear=True)
    ph = synth.slab_phantom()
    beam = synth.pencil_beam(3001, energy=150.0, sigma_cm=0.3)
    whole = oracle.run(db, ph, beam, seed=5, h_begin=7, h_end=3001, track_group=32)
    par = oracle.run_parallel(db, ph, beam, seed=5, h_begin=7, h_end=3001, threads=5, track_group=32)
    assert par.n_histories == whole.n_histories == 2994
    assert par.n_steps == whole.n_steps and par.n_segments == whole.n_segments
    np.testing.assert_allclose(par.edep, whole.edep, rtol=1e-12, atol=1e-9)
    assert abs(par.replayed - whole.replayed) <= 1e-9 * whole.replayed
    assert abs(par.escaped - whole.escaped) <= 1e-9 * max(1.0, whole.escaped)
