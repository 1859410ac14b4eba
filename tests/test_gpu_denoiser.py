"""The learned denoiser end to end at small scale: training pairs from the
engine, training with the library's kernels, and the gain over the plain
method without it on held-out cases (GB300 only)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_denoiser_beats_the_raw_low_history_dose():
    import torch
    from paper_1011_2188_gb300 import denoise, fdc, synth
    eng = fdc.Engine(0)
    eng.load_database(synth.water_database(synth.database_energies(24), 2000, seed=2))
    n_low, n_high, grid = 20_000, 4_000_000, 64
    train = denoise.generate_cases(eng, range(24), n_low, n_high, grid)
    held = denoise.generate_cases(eng, range(5000, 5004), n_low, n_high, grid, keep_phantom=True)
    samples = [denoise.Sample(c.low, c.density, c.high) for c in train]
    net = denoise.UNet(seed=3)
    hist = denoise.train(net, samples, epochs=10, lr=1e-3, lr_final=1e-4, augment=True)
    assert hist[-1] < 0.7 * hist[0], hist
    gains = []
    for c in held:
        s = denoise.Sample(c.low, c.density)
        out = denoise.denoise(net, s)
        g_den = denoise.gamma_pass_rate(c.high, out, (0.2, 0.2, 0.2))
        g_low = denoise.gamma_pass_rate(c.high, c.low, (0.2, 0.2, 0.2))
        gains.append(g_den - g_low)
        # the denoised dose keeps the field's energy (no systematic bias)
        tot = float(out.sum()) / float(c.high.sum())
        assert 0.9 < tot < 1.1, tot
    assert np.mean(gains) > 0.05, gains
    assert min(gains) > 0.0, gains
    eng.close()
