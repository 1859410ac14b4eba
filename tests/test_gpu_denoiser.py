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


def test_committed_weights_reach_the_gamma_floor_on_held_out_cases():
    """The committed U-Net weights on the first five held-out cases of the
    denoiser study (random 128^3 thorax-like phantoms and fields, seeds
    100000-100004, inputs 10^5 histories): 2 %/2 mm gamma against the plain
    10^8-history dose is at least 97 % on every case and 98 % on average
    (the raw 10^5-history dose passes 66-86 %)."""
    import os
    from paper_1011_2188_gb300 import denoise, fdc, synth
    path = os.path.join(os.path.dirname(denoise.__file__), "data", "unet_thorax128.npz")
    eng = fdc.Engine(0)
    eng.load_database(synth.water_database(synth.database_energies(24), 20_000, seed=2))
    net = denoise.UNet(seed=0)
    net.load_npz(path)
    cases = denoise.generate_cases(eng, range(100_000, 100_005), 100_000, 100_000_000, 128, keep_phantom=True)
    g_den, g_low = [], []
    for c in cases:
        out = denoise.denoise(net, denoise.Sample(c.low, c.density))
        g_den.append(denoise.gamma_pass_rate(c.high, out, (0.2, 0.2, 0.2)))
        g_low.append(denoise.gamma_pass_rate(c.high, c.low, (0.2, 0.2, 0.2)))
    print(f"committed weights: gamma denoised {np.round(g_den, 4)}, raw {np.round(g_low, 4)}")
    assert min(g_den) >= 0.97, g_den
    assert np.mean(g_den) >= 0.98, g_den
    assert all(d > l for d, l in zip(g_den, g_low))
    eng.close()
