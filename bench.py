#!/usr/bin/env python
"""Throughput benchmark of the track-repeating dose engine on one GB300.

Workload (default): the thorax-like heterogeneous phantom, 256 x 256 x 128
voxels of 2 mm (lung, soft tissue, bone, air; 4 materials), a water track
database of 24 energies over 70-250 MeV with 10^5 tracks each, and 10^7
protons of 150 MeV (1 % energy spread) over a 10 x 10 cm field.  One step =
one fdc_run of all 10^7 histories (sample, re-trace, tally, dose).

Prints one JSON line: histories/s (value), track-steps/s, the roofline of the
replay kernel, the oracle CPU baseline, end-to-end throughput through the C
ABI with host buffers, and the SM clocks seen during the timed region.

``--impl reference`` times the CPU oracle (the plain sequential FP64 track
repeater) on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "histories/sec and track-steps/sec on 1 GB300; wall time to 2% σ (plain vs denoised)"
# Algorithmic HBM bytes of the replay kernel: the 16-byte step record of each
# replayed step, read once per group of histories sharing the track (16 / G B
# per step for track group G), plus per history its track and start-step
# lookups (step_begin 16, ~9 residual-energy probes 36, tail 8) rounded to 64.
BYTES_PER_RECORD = 16
BYTES_PER_HISTORY = 64
L2_FLUSH_BYTES = 512 << 20
# trained U-Net weights (written by --study denoiser --weights-out)
WEIGHTS = os.path.join(ROOT, "paper_1011_2188_gb300", "data", "unet_thorax128.npz")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fdc", choices=["fdc", "reference"])
    ap.add_argument("--workload", default="thorax", choices=["thorax", "slab", "spots"])
    ap.add_argument("--histories", type=int, default=0, help="override histories per step")
    ap.add_argument("--tracks", type=int, default=100_000, help="database tracks per energy")
    ap.add_argument("--track-group", type=int, default=32,
                    help="histories sharing one database track: 32 (default) is the paper's scheme of "
                         "feeding one history to a thread group; 1 draws a track per history")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--schedule", default="", help="ctas_per_sm,warps_per_cta,chunk,aggregate")
    ap.add_argument("--quick", action="store_true", help="device timing only (sweeps)")
    ap.add_argument("--profile-tracks", type=int, default=10_000,
                    help="database tracks per energy of --study profile_case")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the spot-plan, precision and denoiser measurements of the default line")
    ap.add_argument("--train-cases", type=int, default=200)
    ap.add_argument("--eval-cases", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--variants", type=int, default=1, help="mirror images per training phantom (1-4)")
    ap.add_argument("--no-augment", action="store_true", help="train without the lateral symmetries")
    ap.add_argument("--weights-out", default="", help="save the trained U-Net weights (.npz) to this path")
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--high", type=int, default=100_000_000, help="histories of the target dose")
    ap.add_argument("--study", default="", choices=["", "precision", "denoiser", "unet_timing", "profile_case"],
                    help="precision: FP32 vs FP64 step geometry on the slab phantom, 10^8 histories "
                         "in 100 batches (prints its own JSON line)")
    return ap.parse_args()


def load_peaks(key="hbm_gbs", fallback=6800.0):
    """A measured peak of MEASURED_PEAKS.json (HBM copy GB/s by default; bf16_tflops for the
    dense BF16 burst), else the profiling recipe's fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if key in d:
            return float(d[key]), "measured"
    return fallback, "fallback"


def unet_forward_flops(net, g):
    """Forward FLOPs of one g^3 sample in the direct form of every convolution
    (2 * taps * cin * cout per output voxel; the head counted in full)."""
    out_grid = [g, g, g // 2, g // 2, g // 2, g // 4, g // 4, g // 4, g // 8, g // 8, g // 8,
                g // 4, g // 4, g // 4, g // 2, g // 2, g // 2, g, g, g, g]  # output grid of each layer
    return sum(2.0 * l.k ** 3 * l.cin * l.cout * vox ** 3 for l, vox in zip(net.layers(), out_grid))


def workload(args, world):
    from paper_1011_2188_gb300 import synth
    if args.workload == "thorax":
        n = args.histories or 10_000_000
        db = synth.water_database(synth.database_energies(24), args.tracks, seed=2)
        ph = synth.thorax_phantom(seed=7)
        beam = synth.field_beam(n * world, energy=150.0, width=10.0, height=10.0, sigma_e_rel=0.01)
        desc = ("thorax-like phantom 256x256x128 x 2 mm (air/soft tissue/lung/bone); database 24 energies "
                f"70-250 MeV x {args.tracks} tracks; {n} protons/step, 150 MeV, sigma_E 1%, 10x10 cm field")
    elif args.workload == "slab":
        n = args.histories or 10_000_000
        db = synth.water_database([150.0], 10_000, seed=1)
        ph = synth.slab_phantom()
        beam = synth.pencil_beam(n * world, energy=150.0, sigma_cm=0.3)
        desc = f"water cube 64^3 x 2 mm with 2 cm bone slab; 10^4 tracks at 150 MeV; {n} protons/step, sigma 3 mm"
    else:
        n = args.histories or 20_000_000
        db = synth.water_database(synth.database_energies(24), args.tracks, seed=2)
        ph = synth.slab_phantom()
        beam = synth.spot_plan(seed=11, total=n * world)
        desc = (f"2000 scanning spots in 40 layers 70-230 MeV on the slab phantom; {n} histories/step "
                "(log-normal per spot)")
    return db, ph, beam, n, desc


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9 or p[0] != str(gpu_index):
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(db, ph, beam, seed, h_begin, n, cores):
    """The unchanged oracle on `cores` threads over disjoint, contiguous history
    ranges of [h_begin, h_begin + n) (ctypes releases the GIL around the C
    call; the oracle keeps no global state).  Returns (seconds, track steps)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.lib()
    cuts = [h_begin + (n * i) // cores for i in range(cores + 1)]
    t = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        res = list(ex.map(lambda i: oracle.run(db, ph, beam, seed=seed, h_begin=cuts[i], h_end=cuts[i + 1]),
                          range(cores)))
    return time.perf_counter() - t, sum(r.n_steps for r in res)


def cpu_baseline(db, ph, beam, seed, target_s=8.0):
    """The oracle as it stands on a bounded sample of the workload's histories:
    single-threaded (calibrated to ~target_s seconds), then on every host core
    over disjoint history ranges (~target_s seconds again)."""
    import numpy as np
    import oracle
    oracle.build()
    oracle.run(db, ph, beam, seed=seed, h_begin=0, h_end=200)  # first touch of the inputs, untimed
    # per-history cost from two sizes (a call also has a fixed set-up cost)
    t = time.perf_counter()
    oracle.run(db, ph, beam, seed=seed, h_begin=200, h_end=2200)
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.run(db, ph, beam, seed=seed, h_begin=2200, h_end=22200)
    t2 = time.perf_counter() - t
    per_h = max((t2 - t1) / 18000, t2 / 20000 * 0.1, 1e-7)
    n0 = 22200
    total = int(np.sum(np.asarray(beam["n_histories"], dtype=np.uint64)))  # the sample stays inside the beam
    n = int(min(max(2000, target_s / per_h), 5_000_000, (total - n0) // 4))
    t = time.perf_counter()
    r = oracle.run(db, ph, beam, seed=seed, h_begin=n0, h_end=n0 + n)
    dt = time.perf_counter() - t
    single = {"value": n / dt, "unit": "histories/s", "cores": 1, "kind": "oracle",
              "sample": f"histories [{n0}, {n0 + n}) of the same beam and seed, sequential FP64 oracle",
              "track_steps_per_s": r.n_steps / dt, "seconds": dt}
    cores = host_cores()
    if cores <= 1:
        return single
    m = int(min(n * cores, 20_000_000, total - n0 - n))
    dtp, steps = oracle_parallel(db, ph, beam, seed, n0 + n, m, cores)
    return {"value": m / dtp, "unit": "histories/s", "cores": cores, "kind": "oracle",
            "sample": f"histories [{n0 + n}, {n0 + n + m}) of the same beam and seed; the sequential FP64 "
                      f"oracle on {cores} threads over disjoint contiguous history ranges",
            "track_steps_per_s": steps / dtp, "seconds": dtp, "single_core": single}


def time_to_sigma(eng, beam, ph, seed, target=0.02, n_batches=10, n0=200_000, local=0, track_group=1):
    """Plain method: device time to reach a mean relative batch uncertainty
    (eq. (1)) of ``target`` over voxels above half the maximum dose (Sec. 2.4)
    and, separately, above 0.9 of it (the Bragg-peak region)."""
    from paper_1011_2188_gb300.measure import time_to_sigma as tts
    shape = ph.shape[::-1]
    return {"half_max": tts(eng, beam, shape, seed, target, 0.5, n_batches, n0, local, track_group=track_group),
            "bragg_peak_0.9max": tts(eng, beam, shape, seed, target, 0.9, n_batches, n0, local,
                                     track_group=track_group)}


def denoiser_eval(weights, local=0, n_cases=20, grid=128, n_low=100_000, n_high=100_000_000):
    """The metric's second half (learned denoiser, 128^3 x 2 mm cases): the
    committed U-Net weights on the 20 held-out cases of the denoiser study
    (random thorax-like phantoms and fields, seeds 100000...), each against
    the plain 10^8-history dose by 2 %/2 mm gamma; device time and host wall
    time (beam in host memory to dose in host memory, copies included) of the
    denoised path (10^5-history run + U-Net) and of the plain method run to
    2 % mean uncertainty (eq. (1), D > D_max / 2)."""
    import numpy as np
    from paper_1011_2188_gb300 import denoise, fdc, synth
    if not os.path.exists(weights):
        return {"unavailable": f"no trained weights at {os.path.relpath(weights, ROOT)}"}
    t0 = time.perf_counter()
    eng = fdc.Engine(local)
    db = synth.water_database(synth.database_energies(24), 20_000, seed=2)  # the study's database
    eng.load_database(db)
    net = denoise.UNet(seed=0, device=f"cuda:{local}")
    net.load_npz(weights)
    cases = denoise.generate_cases(eng, range(100_000, 100_000 + n_cases), n_low, n_high, grid, keep_phantom=True)
    rows, summary = denoise.evaluate(net, eng, cases, n_low, (0.2, 0.2, 0.2), host_timing=True)
    eng.close()
    summary["plain_over_denoised_device"] = summary["seconds_plain_2pct"] / summary["seconds_denoised"]
    summary["plain_over_denoised_wall"] = summary["wall_seconds_plain_2pct"] / summary["wall_seconds_denoised"]
    return {"weights": os.path.relpath(weights, ROOT), "grid": grid, "eval_cases": n_cases,
            "histories_low": n_low, "histories_reference": n_high,
            "gamma": "2%/2mm global, threshold 10% of max, against the plain 10^8-history dose",
            "summary": summary,
            "gamma_denoised_per_case": [round(r["gamma_denoised"], 5) for r in rows],
            "seconds": time.perf_counter() - t0}


def spot_plan_bench(eng, local=0, steps=5, seed=21):
    """2000 scanning spots in 40 layers (70-230 MeV, log-normal counts,
    2 x 10^7 histories) on the slab phantom, total plus per-layer dose: one
    persistent launch per run with the autotuned schedule, replayed as a CUDA
    graph (timed with events on the caller's stream around the graph
    launch)."""
    import torch
    from paper_1011_2188_gb300 import synth
    ph = synth.slab_phantom()
    beam = synth.spot_plan(seed=11, total=20_000_000)
    n = int(beam["n_histories"].sum())
    eng.load_phantom(ph)
    eng.set_timing(False)
    sched = eng.autotune(beam, n, seed)
    dev = f"cuda:{local}"
    n_layers = int(beam["layer"].max()) + 1
    dose = torch.empty(ph.shape[::-1], dtype=torch.float64, device=dev)
    ld = torch.empty((n_layers,) + tuple(ph.shape[::-1]), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):  # capture, then relaunches
        eng.run_ex(beam, 0, seed, dose=dose, layer_dose=ld, stream=stream)
    cnt = eng.sync(stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        e0.record(stream)
        eng.run_ex(beam, 0, seed, dose=dose, layer_dose=ld, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    eng.sync(stream)
    t = statistics.median(ms)
    return {"spots": len(beam), "layers": n_layers, "histories": n, "schedule": list(sched),
            "timed": "CUDA graph (memsets, replay, per-layer finalize) relaunched; events around the launch",
            "ms_per_run": t, "histories_per_s": n / (t * 1e-3), "track_steps_per_s": cnt["steps"] / (t * 1e-3)}


def history_vs_batch(eng, beam, ph, n, seed, n_batches=10, local=0, track_group=1):
    """Sec. 2.4 / Fig. 5 analogue on the bench workload: one run of n
    histories in n_batches batches that also keeps the second (squared) tally;
    mean relative uncertainty over D > D_max/2 from eq. (1) and from eq. (2),
    and the device-time cost of keeping the squares (the paper: +18 %)."""
    import torch
    shape = ph.shape[::-1]
    dev = f"cuda:{local}"
    dose = torch.zeros(shape, dtype=torch.float64, device=dev)
    s1, s2, sq = torch.zeros_like(dose), torch.zeros_like(dose), torch.zeros_like(dose)

    def timed(**kw):
        kw["track_group"] = track_group
        eng.run_ex(beam, n, seed, dose=dose, **kw)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = None
        for _ in range(3):
            e0.record()
            eng.run_ex(beam, n, seed, dose=dose, **kw)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    t_plain = timed()
    t_sq = timed(history_sumsq=sq)
    eng.run_ex(beam, n, seed, dose=dose, history_sumsq=sq, n_batches=n_batches, batch_sum=s1, batch_sumsq=s2,
               track_group=track_group)
    eng.sync()
    _, _, rel_b = eng.batch_stats(s1, s2, n_batches, 0.5)
    _, _, rel_h = eng.history_stats(dose, sq, n, 0.5)
    # eq. (2) gives the uncertainty of the mean per-history dose, eq. (1) of
    # the mean batch dose; relative values compare directly
    return {"histories": n, "track_group": track_group, "mean_rel_sigma_batch_eq1": rel_b, "mean_rel_sigma_history_eq2": rel_h,
            "history_over_batch": rel_h / rel_b, "ms_plain": t_plain, "ms_with_squares": t_sq,
            "squares_overhead": t_sq / t_plain - 1.0}


def denoiser_study(args):
    """Learned denoiser: random thorax-like phantoms (grid^3 x 2 mm) and
    random fields; inputs 10^5-history doses (+ density), targets
    high-history doses, all from the engine.  Trains the U-Net with the
    library's kernels and evaluates held-out cases by 2 %/2 mm gamma against
    the high-history plain dose, and by device time against the plain method
    run to 2 % mean uncertainty."""
    import numpy as np
    import torch
    from paper_1011_2188_gb300 import denoise, fdc, synth
    t_all = time.perf_counter()
    eng = fdc.Engine(0)
    db = synth.water_database(synth.database_energies(24), 20_000, seed=2)
    eng.load_database(db)
    n_low = 100_000
    t = time.perf_counter()
    train_cases = denoise.generate_cases(eng, range(args.train_cases), n_low, args.high, args.grid,
                                         variants=args.variants)
    eval_cases = denoise.generate_cases(eng, range(100_000, 100_000 + args.eval_cases), n_low, args.high,
                                        args.grid, keep_phantom=True)
    t_gen = time.perf_counter() - t
    samples = [denoise.Sample(c.low, c.density, c.high) for c in train_cases]
    for c in train_cases:
        c.low = c.high = None
    net = denoise.UNet(seed=0)
    # iteration time
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    denoise.train_step(net, samples[0], 1e-4)
    e1.record()
    e1.synchronize()
    e0.record()
    for i in range(3):
        denoise.train_step(net, samples[i % len(samples)], 1e-4)
    e1.record()
    e1.synchronize()
    it_ms = e0.elapsed_time(e1) / 3
    e0.record()
    for i in range(3):
        denoise.denoise(net, samples[i % len(samples)])
    e1.record()
    e1.synchronize()
    inf_ms = e0.elapsed_time(e1) / 3
    t = time.perf_counter()
    held_out = [denoise.Sample(c.low, c.density, c.high) for c in eval_cases]
    hist, hist_out = denoise.train(net, samples, args.epochs, lr=1e-3, lr_final=5e-5, augment=not args.no_augment,
                                   held_out=held_out)
    del held_out
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    rows, summary = denoise.evaluate(net, eng, eval_cases, n_low, (0.2, 0.2, 0.2))
    g = args.grid
    flops = unet_forward_flops(net, g)
    line = {"study": "denoiser", "grid": g, "train_cases": len(train_cases), "train_phantoms": args.train_cases,
            "eval_cases": args.eval_cases,
            "epochs": args.epochs, "histories_low": n_low, "histories_high": args.high,
            "generate_s": t_gen, "train_s": t_train, "iteration_ms": it_ms, "inference_ms": inf_ms,
            "forward_gflop": flops / 1e9, "inference_tflops": flops / (inf_ms * 1e-3) / 1e12,
            "training_tflops": 3 * flops / (it_ms * 1e-3) / 1e12,
            "augment": not args.no_augment, "loss_history": hist, "held_out_loss_history": hist_out,
            "summary": summary, "cases": rows,
            "note": "doses compared at the low-history count (high-history dose scaled by n_low / n_high)",
            "total_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    if args.weights_out:
        net.save_npz(args.weights_out)


def unet_timing(args):
    print(json.dumps({"study": "unet_timing", **unet_times(args.grid, args.steps, args.warmup)}), flush=True)


def unet_times(g, steps, warmup):
    """Inference and training-step time of the U-Net on one g^3 sample (a
    Gaussian dose on a water grid; the weights do not change the cost), CUDA
    events; inference also replayed as one CUDA graph.  The tensor-core
    roofline takes the model's FLOPs (direct form of every convolution) over
    the graph-replayed inference time against the measured BF16 burst peak."""
    import numpy as np
    import torch
    from paper_1011_2188_gb300 import denoise
    z, y, x = np.meshgrid(*[np.linspace(-1, 1, g)] * 3, indexing="ij")
    dose = torch.from_numpy(np.exp(-(x ** 2 + y ** 2) / 0.1) * (1 + z)).cuda()
    dens = torch.ones((g, g, g), dtype=torch.float32, device="cuda:0")
    s = denoise.Sample(dose, dens, dose)
    net = denoise.UNet(seed=0)
    for _ in range(warmup):
        denoise.denoise(net, s)
        denoise.train_step(net, s, 1e-5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        denoise.denoise(net, s)
    e1.record()
    e1.synchronize()
    inf = e0.elapsed_time(e1) / steps
    e0.record()
    for _ in range(steps):
        denoise.train_step(net, s, 1e-5)
    e1.record()
    e1.synchronize()
    tr = e0.elapsed_time(e1) / steps
    # the same inference replayed as one CUDA graph (no host launch gaps)
    ig = denoise.InferenceGraph(net, s)
    for _ in range(warmup):
        ig.run()
    e0.record()
    for _ in range(steps):
        ig.run()
    e1.record()
    e1.synchronize()
    infg = e0.elapsed_time(e1) / steps
    flops = unet_forward_flops(net, g)
    peak, kind = load_peaks("bf16_tflops", 1900.0)
    achieved = flops / (infg * 1e-3) / 1e12
    return {"grid": g, "inference_ms": inf, "inference_graph_ms": infg, "train_step_ms": tr,
            "forward_gflop": flops / 1e9,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": f"{kind} bf16_tflops (burst)",
                         "count": "model FLOPs of one inference (direct form of every convolution; the "
                                  "upsampling convolutions compute 8/27 of theirs in sub-pixel form)"}}


def precision_case(E, n_total, n_batches=100, n_sub=300_000, local=0):
    """Slab phantom (64^3 x 2 mm, bone slab), pencil beam of energy E:
    n_total histories in n_batches batches with FP32 and with FP64 step
    geometry; FP32 vs FP64 dose on the device, both against the FP64 oracle on
    the first n_sub histories (threaded over disjoint history ranges),
    per-voxel batch uncertainty from the FP64 batch sums (eq. (1)), and the
    device time to 2 % mean uncertainty in the Bragg-peak region."""
    import numpy as np
    import torch
    import oracle
    from paper_1011_2188_gb300 import fdc, synth
    oracle.build()
    db = synth.water_database([E], 10_000, seed=1)
    ph = synth.slab_phantom()
    beam = synth.pencil_beam(n_total, energy=E, sigma_cm=0.3)
    eng = fdc.Engine(local)
    eng.load_database(db)
    eng.load_phantom(ph)
    shape = ph.shape[::-1]
    dev = f"cuda:{local}"
    out = {"energy_mev": E, "histories": n_total, "n_batches": n_batches}
    doses = {}
    for fp64 in (False, True):
        s1 = torch.zeros(shape, dtype=torch.float64, device=dev)
        s2 = torch.zeros_like(s1)
        dose = torch.zeros_like(s1)
        eng.run_ex(beam, n_total, 5, n_batches=n_batches, batch_sum=s1, batch_sumsq=s2, dose=dose,
                   fp64_geometry=fp64)
        eng.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        eng.run_ex(beam, n_total, 5, n_batches=n_batches, batch_sum=s1, batch_sumsq=s2, dose=dose,
                   fp64_geometry=fp64)
        e1.record()
        e1.synchronize()
        cnt = eng.sync()
        mean, sigma, rel_half = eng.batch_stats(s1, s2, n_batches, 0.5)
        _, _, rel_peak = eng.batch_stats(s1, s2, n_batches, 0.9)
        key = "fp64" if fp64 else "fp32"
        sec = e0.elapsed_time(e1) * 1e-3
        # histories to reach 2 % in the Bragg-peak region, from sigma ~ N^-1/2
        n2 = n_total * (rel_peak / 0.02) ** 2
        out[key] = {"seconds": sec, "histories_per_s": n_total / sec,
                    "track_steps_per_s": cnt["steps"] / sec,
                    "mean_rel_sigma_half_max": rel_half, "mean_rel_sigma_peak_0.9max": rel_peak,
                    "histories_for_2pct_peak": n2, "seconds_for_2pct_peak": sec * n2 / n_total}
        doses[key] = dose.cpu().numpy()
    d32, d64 = doses["fp32"], doses["fp64"]
    mx = d64.max()
    out["fp32_vs_fp64_device"] = {"max_abs_over_max": float(np.abs(d32 - d64).max() / mx),
                                  "mean_abs_over_max": float(np.abs(d32 - d64).mean() / mx)}
    ref = oracle.run_parallel(db, ph, beam, seed=5, h_begin=0, h_end=n_sub)
    d_ref = oracle.dose(ph, ref.edep)
    sub = {"histories": n_sub}
    for fp64 in (False, True):
        d = torch.zeros(shape, dtype=torch.float64, device=dev)
        eng.run_ex(beam, n_sub, 5, dose=d, fp64_geometry=fp64)
        eng.sync()
        dd = d.cpu().numpy()
        sub["fp64" if fp64 else "fp32"] = {
            "max_abs_over_max": float(np.abs(dd - d_ref).max() / d_ref.max()),
            "mean_abs_over_max": float(np.abs(dd - d_ref).mean() / d_ref.max()),
            "total_energy_rel": float(abs(dd.sum() - d_ref.sum()) / d_ref.sum())}
    out["vs_oracle"] = sub
    eng.close()
    return out


def precision_study(args):
    """Precision study (10^8 histories in 100 batches, FP32 vs FP64 step
    geometry vs the FP64 oracle) at 150 MeV and at the paper's 121 MeV."""
    n_total = args.histories or 100_000_000
    res = {"study": "precision", "histories": n_total, "n_batches": 100}
    for E in (150.0, 121.0):
        res[f"{E:g}MeV"] = precision_case(E, n_total)
    print(json.dumps(res), flush=True)


def profile_case(args):
    """Small cases for ncu captures (the full-size workload holds ~13 GB on
    the device): the thorax phantom with a 24 x --profile-tracks database
    (default 10^4: 4.6 x 10^7 step records, 1.3 GB), --histories (default
    10^6) over the 10 x 10 cm field with 32 histories per track, replayed
    twice (capture the second launch); then one launch of the atomic probe
    (2^28 updates over 64 MB).  Prints the replay's counters so per-step
    figures can be formed."""
    import torch
    from paper_1011_2188_gb300 import fdc, synth
    n = args.histories or 1_000_000
    db = synth.water_database(synth.database_energies(24), args.profile_tracks, seed=2)
    ph = synth.thorax_phantom(seed=7)
    beam = synth.field_beam(n, energy=150.0, width=10.0, height=10.0, sigma_e_rel=0.01)
    eng = fdc.Engine(0)
    eng.load_database(db)
    eng.load_phantom(ph)
    dose = torch.empty(ph.shape[::-1], dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        eng.run_ex(beam, n, 1234, dose=dose, track_group=args.track_group, graph=False)
        cnt = eng.sync()
    slots = torch.zeros(1 << 23, dtype=torch.int64, device="cuda:0")
    ms = fdc.probe_atomics(slots, 1 << 28)
    eng.close()
    print(json.dumps({"study": "profile_case", "histories": n, "tracks_per_energy": args.profile_tracks,
                      "track_group": args.track_group,
                      "steps": cnt["steps"], "segments": cnt["segments"], "probe_ops": 1 << 28,
                      "probe_ms": ms, "kernel_source_sha16": kernel_source_hash()}), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    db, ph, beam, n, desc = workload(args, 1)
    import oracle
    oracle.build()
    oracle.run(db, ph, beam, seed=1234, h_begin=0, h_end=200)  # first touch of the inputs, untimed
    # per-history cost from two sizes (a call also has a fixed set-up cost)
    t = time.perf_counter()
    oracle.run(db, ph, beam, seed=1234, h_begin=200, h_end=1200)
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.run(db, ph, beam, seed=1234, h_begin=1200, h_end=11200)
    t2 = time.perf_counter() - t
    per_h = max((t2 - t1) / 9000, t2 / 10000 * 0.1, 1e-7)
    cores = host_cores()
    total = int(sum(int(x) for x in beam["n_histories"]))
    per = int(max(1000, min(8.0 / per_h, (total - 11200) // (2 * cores))))  # ~8 s per thread and step
    off = 11200

    def next_range():  # consecutive history ranges of the beam, wrapping inside it
        nonlocal off
        if off + per * cores > total:
            off = 11200
        h0 = off
        off += per * cores
        return h0

    for _ in range(args.warmup):
        oracle.run(db, ph, beam, seed=1234, h_begin=off, h_end=off + min(per, 2000))
    # each step: per histories on every host core, over disjoint history ranges
    times, steps = [], 0
    for _ in range(args.steps):
        dt, st = oracle_parallel(db, ph, beam, 1234, next_range(), per * cores, cores)
        times.append(dt)
        steps += st
    tot = sum(times)
    value = per * cores * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "histories/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "histories_per_step": per * cores},
        "track_steps_per_s": steps / tot,
        "cpu_baseline": {"value": value, "unit": "histories/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per * cores} histories per step of the workload; the sequential FP64 "
                                   f"oracle on {cores} threads over disjoint contiguous history ranges"},
        "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_source_hash():
    """Hash of the replay kernel's sources: a DRAM-traffic figure measured on
    one version of the kernel is reported only for that version."""
    import hashlib
    h = hashlib.sha256()
    for f in ("fdc_kernels.cu", "fdc_internal.h"):
        with open(os.path.join(ROOT, "paper_1011_2188_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic_per_step():
    """DRAM bytes (read + write) per replayed track step of the replay kernel
    from the committed ncu summary, if it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", "replay_kernel_dram_per_step.txt")
    if not os.path.exists(path):
        return None, "no capture summary"
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha16") != kernel_source_hash():
        return None, "kernel changed since the capture"
    return float(kv["dram_bytes_per_step"]), kv.get("workload", "")


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.study == "precision":
        if rank == 0:
            precision_study(args)
        return
    if args.study == "denoiser":
        if rank == 0:
            denoiser_study(args)
        return
    if args.study == "unet_timing":
        if rank == 0:
            unet_timing(args)
        return
    if args.study == "profile_case":
        if rank == 0:
            profile_case(args)
        return

    import numpy as np
    import torch
    from paper_1011_2188_gb300 import build as fdc_build
    fdc_build.build()
    from paper_1011_2188_gb300 import fdc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        # one rank per GPU; the ranks' int64 tallies are summed over NCCL
        os.environ.setdefault("NCCL_DEBUG", "INFO")
        os.environ.setdefault("NCCL_DEBUG_SUBSYS", "INIT")
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    db, ph, beam, n, desc = workload(args, world)
    eng = fdc.Engine(local)
    t_load = time.perf_counter()
    eng.load_database(db)
    eng.load_phantom(ph)
    t_load = time.perf_counter() - t_load
    seed = 1234
    from paper_1011_2188_gb300.shard import weak_shard
    offset, _ = weak_shard(n, rank)
    sched = None
    if args.schedule:
        sched = tuple(int(x) for x in args.schedule.split(","))
    if args.autotune:
        sched = eng.autotune(beam, min(n, 1_000_000), seed, history_offset=offset, track_group=args.track_group)
    dev = f"cuda:{local}"
    dose = torch.empty(ph.shape[::-1], dtype=torch.float64, device=dev)
    tally = torch.empty(ph.shape[::-1], dtype=torch.int64, device=dev) if world > 1 else None
    layer_dose = None
    if args.workload == "spots":  # total dose plus the dose of every energy layer
        n_layers = int(beam["layer"].max()) + 1
        layer_dose = torch.empty((n_layers,) + tuple(ph.shape[::-1]), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    eng.set_timing(True)

    def one_step():
        if world == 1:
            eng.run_ex(beam, n, seed, history_offset=offset, dose=dose, layer_dose=layer_dose, stream=stream,
                       schedule=sched, track_group=args.track_group)
        else:
            # this rank's histories into its int64 tally, the exact sum over
            # the ranks (Sec. 2.3: the two GPUs' doses summed at the end),
            # then the dose of the whole job
            eng.run_ex(beam, n, seed, history_offset=offset, tally=tally, stream=stream,
                       schedule=sched, track_group=args.track_group)
            dist.all_reduce(tally)
            eng.dose_from_tally(tally, dose, stream=stream)

    for _ in range(max(args.warmup, 0)):
        one_step()
    cnt = eng.sync(stream)
    steps_per_run = cnt["steps"]
    segs_per_run = cnt["segments"]
    hist_per_run = cnt["histories"]
    assert hist_per_run == n

    # ---- device-resident timing
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    step_ms, replay_ms = [], []
    for _ in range(args.steps):
        flush.zero_()                          # L2 flush between timed steps
        ev0.record(stream)
        one_step()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        replay_ms.append(eng.last_kernel_ms()[0])
    torch.cuda.synchronize()
    clk = clocks.stop(local)
    if dist:
        dist.barrier()
    cnt = eng.sync(stream)
    ms = sum(step_ms) / len(step_ms)
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t[0])
    value = n * world / (ms * 1e-3)
    rep_ms = statistics.median(replay_ms)
    if args.quick:
        if rank == 0:
            print(json.dumps({"value": value, "ms_per_step": ms, "replay_ms": rep_ms, "schedule": sched,
                              "tracks": args.tracks, "track_group": args.track_group,
                              "track_steps_per_s": steps_per_run * world / (ms * 1e-3), "clocks": clk,
                              "flags": os.environ.get("FDC_NVCC_FLAGS", "")}), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    # ---- ablation: a separate track per history (Sec. 4: +50 % time on the GTX 295)
    indep = None
    if args.track_group != 1 and world == 1:
        t_ind = []
        for i in range(3 + 3):
            ev0.record(stream)
            eng.run_ex(beam, n, seed, history_offset=offset, dose=dose, layer_dose=layer_dose, stream=stream,
                       schedule=sched, track_group=1)
            ev1.record(stream)
            ev1.synchronize()
            if i >= 3:
                t_ind.append(ev0.elapsed_time(ev1))
        ms_ind = sum(t_ind) / len(t_ind)
        indep = {"track_group": 1, "histories_per_s": n / (ms_ind * 1e-3), "ms_per_step": ms_ind,
                 "time_ratio_vs_shared": ms_ind / ms}

    # ---- end to end through the C ABI with host buffers (beam in, dose out)
    host_dose = torch.empty(ph.shape[::-1], dtype=torch.float64).pin_memory().numpy()
    e2e_times = []
    sub = beam.copy()
    for i in range(max(2, min(args.steps, 5))):
        t = time.perf_counter()
        eng.run_host(sub, n, seed + 1 + i, host_dose, track_group=args.track_group)
        e2e_times.append(time.perf_counter() - t)
    e2e_s = statistics.median(e2e_times[1:])
    h2d = int(fdc.SPOT_DTYPE.itemsize * len(beam) + 8 * (len(beam) + 1))
    d2h = int(host_dose.nbytes)

    # ---- L2 atomic probe (denominator of the tally-update roofline)
    slots = torch.zeros(1 << 23, dtype=torch.int64, device=dev)  # 64 MB, like the tally
    n_ops = 1 << 31
    fdc.probe_atomics(slots, n_ops // 8)  # warm-up
    atom_ms = min(fdc.probe_atomics(slots, n_ops) for _ in range(3))
    atom_peak = n_ops / (atom_ms * 1e-3)

    hbm_peak, peak_kind = load_peaks()
    # algorithmic HBM bytes of one replay launch: the step records (16 B per
    # replayed step, shared by the G histories of a track group), and, as a
    # second count, the same plus every history's track and start-step lookups
    rec_bytes = BYTES_PER_RECORD * steps_per_run / max(1, args.track_group)
    alg_bytes = rec_bytes
    alg_bytes_lookups = rec_bytes + BYTES_PER_HISTORY * hist_per_run
    achieved = alg_bytes / (rep_ms * 1e-3) / 1e9
    achieved_lookups = alg_bytes_lookups / (rep_ms * 1e-3) / 1e9
    atom_achieved = segs_per_run / (rep_ms * 1e-3)
    per_step, traffic_src = measured_traffic_per_step()
    traffic = per_step * steps_per_run if per_step is not None and args.workload == "thorax" else None

    line = {
        "metric": METRIC, "value": value, "unit": "histories/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "histories_per_step": n, "tally": "int64 fixed point 2^-28 MeV",
                   "l2": "flushed between timed steps (512 MB write); track working set > L2",
                   "schedule": list(sched) if sched else "default",
                   "parallelism": "history ranges per rank, int64 tally all-reduce (NCCL)" if world > 1
                   else "one GPU", "track_group": args.track_group},
        "track_steps_per_s": steps_per_run * world / (ms * 1e-3),
        "segments_per_s": segs_per_run * world / (ms * 1e-3),
        "steps_per_history": steps_per_run / hist_per_run,
        "replay_ms": rep_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "algorithmic_count": f"{BYTES_PER_RECORD} B per replayed step / track group "
                                          f"({args.track_group})",
                     "with_history_lookups": {"bytes_per_launch": alg_bytes_lookups, "achieved": achieved_lookups,
                                              "frac": achieved_lookups / hbm_peak,
                                              "count": f"+ {BYTES_PER_HISTORY} B per history"},
                     "traffic_source": traffic_src,
                     "note": "not the binding resource: the replay kernel is bound by instruction issue "
                             "(ncu issue-slot utilisation) and L2 atomics (roofline_l2_atomic)"},
        "roofline_l2_atomic": {"achieved": atom_achieved, "peak": atom_peak, "unit": "atomic/s",
                               "frac": atom_achieved / atom_peak,
                               "note": "one tally update per voxel segment; peak from the hashed int64 "
                                       "atomic probe on this GPU (random 8-byte slots of a 64 MB array)"},
        "e2e": {"value": n / e2e_s, "unit": "histories/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": (2 if world == 1 else 3) * args.steps,
        "ablation_independent_tracks": indep,
        "clocks": clk,
        "load_s": t_load,
    }
    if rank == 0 and args.workload != "spots":  # batches of a spot plan would cover different spots
        line["time_to_2pct_sigma_plain"] = time_to_sigma(eng, beam, ph, seed + 99, local=local,
                                                         track_group=args.track_group)
        line["history_by_history"] = history_vs_batch(eng, beam, ph, n, seed + 7, local=local,
                                                      track_group=args.track_group)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(db, ph, beam, seed)
    if rank == 0 and args.workload == "thorax" and world == 1 and not args.no_extras:
        # the other configurations, each timed on its own (not part of `value`)
        line["spot_plan_2000"] = spot_plan_bench(eng, local=local)
        eng.close()
        eng = None
        line["precision_fp32_fp64"] = precision_case(150.0, 100_000_000, local=local)
        line["denoiser"] = denoiser_eval(WEIGHTS, local=local)
        line["denoiser"]["unet_128"] = unet_times(128, 20, 3)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if eng is not None:
        eng.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
