#!/usr/bin/env python
"""Benchmark of the NARVis hot path on one GB300: a 350M-point trajectory scene (1M particles x
350 RK4 steps, K = 3 attributes) rendered at 1920x1080 -- render + resolve/pack passes of the
rasterizer and the U-Net forward -- reported as points/s (and frames/s).

    python bench.py [--steps K] [--warmup W] [--prec bf16|fp32] [--impl ours|reference]

One step = one whole frame through nrv_render_batch with the scene resident in HBM.  `value`
is points/s = N * frames/s over all ranks (replicas: each rank renders the frame).  `e2e`
measures the same through the public API per frame: the camera goes in from the host and the
RGB frame comes back to pinned host memory inside the timed region.  The reference arm
(--impl reference) times the CPU oracle on the host cores on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
BYTES_PER_POINT = 12.0          # xyz read once per frame for every view
# DRAM bytes the render pass of the 350M-point 1080p trajectory frame moves (one ncu capture of
# its seven launches: every chunk box, the sub-chunk boxes of surviving chunks, the positions of
# the prepass chunks and of the surviving sub-chunks, tile-bound reads, atomics)
RENDER_TRAFFIC_BYTES = 1.2343e9
# host -> device bytes of one replayed nrv_render_batch frame: the library's table of the views
# (8 slots of 88 bytes and a count, 712 bytes), copied whole whatever the view count
VIEW_TABLE_BYTES = 712


def network_floor_ms(H, W, c0, hbm_gbs, tflops):
    """Lower bound of one U-Net forward at H x W: per layer the larger of its FLOP time at the
    tensor peak and its byte time at the HBM peak (each layer reads its inputs and writes its
    output once, BF16; the input G-buffer is 8 channels; the head is fused into the last conv,
    which writes FP32 RGB instead of its activations)."""
    Hp, Wp = H + (-H) % 8, W + (-W) % 8
    px = [Hp * Wp // 4 ** l for l in range(4)]
    ch = [16, 32, 64, 128]
    layers = []                       # (flops, bytes)

    def conv(cin, cout, n, cin_bytes=None, out_bytes=None):
        layers.append((2.0 * 9 * cin * cout * n,
                       n * ((cin_bytes if cin_bytes is not None else 2 * cin) +
                            (out_bytes if out_bytes is not None else 2 * cout))))

    conv(c0, 16, px[0], cin_bytes=16)                       # e0a: 8 BF16 input channels
    conv(16, 16, px[0])                                     # e0b
    for l in range(1, 4):
        layers.append((0.0, px[l] * 2 * ch[l - 1] * 5))     # 2x2 average pool
        conv(ch[l - 1], ch[l], px[l])
        conv(ch[l], ch[l], px[l])
    for l in (3, 2, 1):
        layers.append((2.0 * ch[l] * 4 * ch[l - 1] * px[l],  # transposed conv
                       px[l] * 2 * ch[l] + px[l - 1] * 2 * ch[l - 1]))
        conv(2 * ch[l - 1], ch[l - 1], px[l - 1])
        if l > 1:
            conv(ch[l - 1], ch[l - 1], px[l - 1])
    conv(16, 16, px[0], out_bytes=12)                        # d0b + head: FP32 RGB
    layers.append((2.0 * 16 * 3 * px[0], 0.0))
    return sum(max(f / (tflops * 1e12), b / (hbm_gbs * 1e9)) for f, b in layers) * 1e3


def gated_flops_per_frame(H, W, c0):
    """FLOPs of one forward of the gated network at H x W (canvas padded to multiples of 8):
    per gated 3x3 conv 2 * 9 * C_in * (2 C_out) per output pixel (feature and gate), per
    transposed conv 2 * C_in * 4 * C_out per input pixel, the 1x1 layers 2 * C_in * C_out."""
    from oracle import gated
    Hp, Wp = H + (-H) % 8, W + (-W) % 8
    px = [Hp * Wp // 4 ** l for l in range(4)]
    level = {"inj": 0, "e0": 0, "e1": 1, "e2": 2, "e3": 3, "up2": 3, "d2": 2, "up1": 2, "d1": 1,
             "up0": 1, "d0": 0, "head": 0}
    f = 0.0
    for name, kind, ci, co in gated.layers(c0):
        n = px[level[name]]
        f += {"gated": 2.0 * 9 * ci * 2 * co, "convT2": 2.0 * ci * 4 * co, "conv1": 2.0 * ci * co}[kind] * n
    return f


def gated_params(c0, seed=1):
    """Seeded Xavier-uniform weights, zero biases, in the gated network's flat layout."""
    import numpy as np
    import nrv_inputs as I
    from oracle import gated
    flat = []
    for t, (name, kind, ci, co) in enumerate(gated.layers(c0)):
        for k, shp in enumerate(gated.shapes(kind, ci, co)):
            if len(shp) == 1:
                flat.append(np.zeros(shp, np.float32))
            else:
                k2 = 9 if kind == "gated" else (4 if kind == "convT2" else 1)
                flat.append(I.xavier_uniform(seed, 2000 + 8 * t + k, shp, ci * k2, co * k2).ravel())
    return np.concatenate(flat).astype(np.float32)


def measure_local_peaks(dev):
    """Peaks the measured-peaks file does not hold, measured on this GPU with the library's
    probes: FP32 FMA throughput (the FP32 network's roofline), random 64-bit atomicMin on a
    16.6 MB (one 1080p key image, L2-resident) buffer (the depth test's), and an FP8 GEMM
    through cuBLASLt (torch._scaled_mm; None where unavailable)."""
    import torch
    from paper_2407_19097_gb300 import nrv
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def timed_ms(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    blocks, iters = sms * 8, 2048
    out = torch.empty(blocks * 256, device=dev)
    ms = timed_ms(lambda: nrv.check(nrv.lib().nrv_probe_ffma(nrv._ptr(out), blocks, iters, nrv._stream())))
    ffma = 16.0 * iters * blocks * 256 / (ms * 1e-3) / 1e12
    words, ops = 1920 * 1080, 1 << 26
    buf = torch.zeros(words, dtype=torch.int64, device=dev)
    ms = timed_ms(lambda: nrv.check(nrv.lib().nrv_probe_atomic_min(nrv._ptr(buf), words, ops, 7,
                                                                    nrv._stream())))
    atom = ops / (ms * 1e-3) / 1e9
    fp8 = None
    try:
        n = 8192
        a8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        ms = timed_ms(lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one,
                                               out_dtype=torch.bfloat16), reps=20)
        fp8 = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
    except Exception:
        fp8 = None
    return {"fp32_ffma_tflops": ffma, "atomic64_min_g_per_s_l2": atom, "fp8_gemm_tflops": fp8,
            "note": "measured in this run: FFMA probe (8 independent chains per thread), "
                    "random 64-bit atomicMin over 2.07M words, cuBLASLt FP8 e4m3 8192^3"}


def job_rate(ms, units_per_rank, world, device=None):
    """Whole-job throughput of `world` replicas: the slowest rank's time per step (max over
    ranks; every rank must call this) and units_per_rank * world / that time, per second."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--particles", type=int, default=1_000_000)
    ap.add_argument("--steps-per-particle", type=int, default=350)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--c5-steps", type=int, default=2000)
    ap.add_argument("--sparsity", default="1,2,4,10",
                    help="c5: subsampling factors of the sparsity study (Tab. 6)")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-fp8", action="store_true")
    ap.add_argument("--no-gated", action="store_true")
    ap.add_argument("--terrain-grid", type=int, default=14142,
                    help="c4: terrain points per side (14142: 200M points; smaller for profiling)")
    ap.add_argument("--config", default="c3", choices=["c3", "c2", "c4", "c5", "train"],
                    help="c3 (default): the 350M-point trajectory frame; c2: 50M-point vortex grid "
                         "frame with network precision vs FP64; c4: 200M-point terrain, 8 views of "
                         "uneven size in one batch; c5: training step time and held-out quality; "
                         "train: the training step alone on seeded inputs of c5's shape")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clock/throttle samples every 10 ms while the timed region runs.  start() returns
    once the first sample has been written (nvidia-smi takes a while to come up), so that a short
    timed region is still covered."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(tempfile.gettempdir(), f"nrv_clocks_{os.getpid()}_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        self.skip = os.path.getsize(self.path)  # samples taken before the timed region are not used

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.close()
        mhz, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            f.seek(getattr(self, "skip", 0))
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) < 9:
                    continue
                try:
                    mhz.append(float(t[1]))
                    mx.append(float(t[2]))
                except ValueError:
                    continue
                for n, v in zip(names, t[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(mhz)}


def make_workload(a):
    import nrv_inputs as I
    t0 = time.time()
    sc = I.trajectory_scene(a.particles, a.steps_per_particle, seed=2)
    view = I.fitted_view(sc, a.width, a.height)
    ds, do = I.depth_normalisation(sc, view)
    return sc, view, ds, do, time.time() - t0


def workload_name(a):
    return (f"trajectories {a.particles}x{a.steps_per_particle} = "
            f"{a.particles * a.steps_per_particle} points, K=3, {a.width}x{a.height}")


def unet_params(c0, seed=1):
    import numpy as np
    import nrv_inputs as I
    from paper_2407_19097_gb300 import nrv
    flat = np.zeros(nrv.param_count(c0), np.float32)
    for t, (name, kind, ci, co, wo, bo) in enumerate(nrv.layer_table(c0)):
        k2 = {0: 9, 1: 4, 2: 1}[kind]
        shape = {0: (co, ci, 3, 3), 1: (ci, co, 2, 2), 2: (co, ci)}[kind]
        flat[wo:wo + int(np.prod(shape))] = I.xavier_uniform(seed, 1000 + t, shape, ci * k2,
                                                             co * k2).ravel()
    return flat


def oracle_frame(sc, view, ds, do, max_seconds=None):
    """The CPU oracle on one frame: render + resolve (C, one thread), pack, FP64 U-Net (numpy,
    BLAS threads).  Returns (seconds, rgb float64 [H,W,3], seconds of the raster part)."""
    import numpy as np
    import oracle
    from oracle import unet
    c0 = len(sc.channels) + 2
    t0 = time.perf_counter()
    key, d, m, g = oracle.rasterize(sc, view)
    hn, wn = (view.height + 7) // 8 * 8, (view.width + 7) // 8 * 8
    x = oracle.pack(d, m, g, sc.channels, ds, do, hn, wn, 8, 0)
    t1 = time.perf_counter()
    y = unet.forward(x[None, :, :, :c0].astype(np.float64), unet.unflatten(unet_params(c0), c0))[0]
    t2 = time.perf_counter()
    return t2 - t0, y[:view.height, :view.width], t1 - t0


REFERENCE_BUDGET_S = 150.0   # the whole --impl reference run (warm-up and timed steps)


def oracle_sample(sc, view, ds, do, step, frac, band_rows):
    """One bounded sample of a frame on the CPU oracle: render + resolve + pack of a contiguous
    fraction `frac` of the points (C, all cores) and the FP64 U-Net on a band_rows-row band of
    the packed frame (numpy, all BLAS threads).  Returns (seconds the sample took, the
    whole-frame time it extrapolates to)."""
    import numpy as np
    import oracle
    from oracle import unet
    c0 = len(sc.channels) + 2
    n = max(1, int(sc.n * frac))
    lo = (step * n) % max(1, sc.n - n + 1)
    part = sc.subset(np.arange(lo, lo + n))
    hn, wn = (view.height + 7) // 8 * 8, (view.width + 7) // 8 * 8
    t0 = time.perf_counter()
    key = oracle.visibility(part.xyz, view, threads="all")
    d, m, g = oracle.resolve(key, part.attr, part.n_words)
    x = oracle.pack(d, m, g, sc.channels, ds, do, hn, wn, 8, 0)
    t1 = time.perf_counter()
    r0 = (step * band_rows) % (hn - band_rows + 1) // 8 * 8
    unet.forward(x[None, r0:r0 + band_rows, :, :c0].astype(np.float64),
                 unet.unflatten(unet_params(c0), c0))
    t2 = time.perf_counter()
    return t2 - t0, (t1 - t0) * (sc.n / n) + (t2 - t1) * hn / band_rows


def run_reference(a, rank, world):
    """Reference arm: the CPU oracle on the host cores, same workload and metric.  Each step is
    a bounded sample of the frame -- a fraction of the points and a band of the network rows,
    sized so that all warm-up and timed steps take about REFERENCE_BUDGET_S -- and the line's
    value is the whole-frame rate the samples extrapolate to; ms_per_step is the time a sample
    actually took."""
    if rank != 0:
        return
    sc, view, ds, do, gen_s = make_workload(a)
    per_step = REFERENCE_BUDGET_S / max(1, a.warmup + a.steps)
    # about 7 s per whole frame on 16 cores (0.3 s render pass, the rest the FP64 network):
    # scale both parts by the step's share of that
    share = min(1.0, per_step / 7.0)
    hn = (view.height + 7) // 8 * 8
    band = max(8, min(hn, int(hn * share) // 8 * 8))
    frac = max(1e-3, min(1.0, share))
    took, frames = [], []
    for i in range(a.warmup + a.steps):
        t, f = oracle_sample(sc, view, ds, do, i, frac, band)
        if i >= a.warmup:
            took.append(t)
            frames.append(f)
    sec = sum(frames) / len(frames)
    v = sc.n / sec
    ncpu = os.cpu_count()
    sample = (f"per step: render+resolve+pack of {frac:.4f} of the points in C on all cores, FP64 "
              f"U-Net on a {band}-row band of the {hn}-row frame in numpy on all BLAS threads; the "
              f"value is the whole-frame rate these samples extrapolate to ({sec:.2f} s per frame)")
    line = {"impl": "reference", "metric": "points/s (frames/s) at 1080p", "value": v,
            "unit": "points/s", "n_gpus": 0, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * sum(took) / len(took), "extrapolated_frame_ms": sec * 1e3,
            "fps": 1.0 / sec, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 raster / f64 net",
            "data": "synthetic", "config": {"workload": workload_name(a)},
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": ncpu, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _events_ms(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _quality(got, ref):
    import numpy as np
    r = float(ref.max() - ref.min())
    mse = float(np.mean((got - ref) ** 2))
    return {"psnr_db": 10 * np.log10(r * r / mse) if mse > 0 else None,
            "max_abs": float(np.abs(got - ref).max())}


def run_c2(a):
    """50M-point jittered vortex grid (K = 5), one 1080p view: render + resolve + pack rate, and
    the network in FP32, BF16 and FP8 -- time and error against the FP64 oracle on this frame."""
    import numpy as np
    import torch
    import nrv_inputs as I
    from oracle import unet
    import oracle
    from paper_2407_19097_gb300 import nrv
    dev = torch.device("cuda", 0)
    t0 = time.time()
    sc = I.vortex_grid_scene(368, seed=1)
    view = I.cube_view(1920, 1080)
    ds, do = I.depth_normalisation(sc, view)
    gen_s = time.time() - t0
    c0 = len(sc.channels) + 2
    scene = nrv.Scene(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.attr.view(np.int32)).to(dev),
                      sc.n_words)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(unet_params(c0)).to(dev))
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    H, W = view.height, view.width
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for name, prec in (("fp32", nrv.PREC_F32), ("bf16", nrv.PREC_BF16)):
        nrv.set_profiling(True)
        ms = _events_ms(lambda: nrv.render_batch(scene, net, desc, [view], [rgb], prec), a.steps, a.warmup,
                        stream)
        nrv.set_profiling(False)
        st = nrv.timings()
        out[name] = {"frame_ms": ms, "render_ms": st[1], "resolve_pack_ms": st[2], "network_ms": st[3],
                     "rgb": rgb.float().cpu().numpy().astype(np.float64)}
    # FP8, calibrated on this frame's BF16 input
    key = torch.empty((H, W), dtype=torch.int64, device=dev)
    dpl = torch.empty((H, W), dtype=torch.int32, device=dev)
    msk = torch.empty((H, W), dtype=torch.uint8, device=dev)
    gat = torch.empty((sc.n_words, H, W), dtype=torch.int32, device=dev)
    nrv.rasterize(scene, [view], [key], [dpl], [msk], [gat])
    xb = torch.empty(((H + 7) // 8 * 8, (W + 7) // 8 * 8, 8), dtype=torch.bfloat16, device=dev)
    nrv.pack(dpl, msk, gat, H, W, desc, nrv.PREC_BF16, xb)
    net.calibrate(xb, 1, H, W)
    inv8 = 1.0 / net.act_scales()[0]
    nrv.set_profiling(True)
    ms8 = _events_ms(lambda: nrv.render_batch(scene, net, desc, [view], [rgb], nrv.PREC_FP8_E4M3, inv8),
                     a.steps, a.warmup, stream)
    nrv.set_profiling(False)
    st = nrv.timings()
    out["fp8_e4m3"] = {"frame_ms": ms8, "render_ms": st[1], "resolve_pack_ms": st[2],
                       "network_ms": st[3], "rgb": rgb.float().cpu().numpy().astype(np.float64)}
    # NRV_PREC_FP8: E4M3 for levels 1-3, BF16 for level 0
    nrv.set_profiling(True)
    ms8m = _events_ms(lambda: nrv.render_batch(scene, net, desc, [view], [rgb], nrv.PREC_FP8),
                      a.steps, a.warmup, stream)
    nrv.set_profiling(False)
    st = nrv.timings()
    out["fp8"] = {"frame_ms": ms8m, "render_ms": st[1], "resolve_pack_ms": st[2],
                        "network_ms": st[3], "rgb": rgb.float().cpu().numpy().astype(np.float64)}
    # the FP64 oracle frame
    _, d, m, g = oracle.rasterize(sc, view)
    hn, wn = (H + 7) // 8 * 8, (W + 7) // 8 * 8
    x = oracle.pack(d, m, g, sc.channels, ds, do, hn, wn, 8, 0)
    y = unet.forward(x[None, :, :, :c0].astype(np.float64), unet.unflatten(unet_params(c0), c0))[0][:H, :W]
    line = {"config": "c2", "metric": "points/s (frames/s) at 1080p",
            "workload": f"vortex grid 368^3 = {sc.n} points, K=5, 1920x1080", "data": "synthetic",
            "value": sc.n / (out["bf16"]["frame_ms"] * 1e-3), "unit": "points/s",
            "render_points_per_s": sc.n / ((out["bf16"]["render_ms"] + out["bf16"]["resolve_pack_ms"]) * 1e-3),
            "scene_gen_s": gen_s}
    for k, v in out.items():
        line[k] = {kk: vv for kk, vv in v.items() if kk != "rgb"}
        line[k]["vs_fp64"] = _quality(v["rgb"], y)
    print(json.dumps(line), flush=True)


def run_c4(a):
    """200M-point terrain (RGB u8x4 + intensity), 8 views of uneven size (2 x 2160^2 stereo,
    4 x 1920x1080, 2 x 960x540) rendered and shaded in one nrv_render_batch call."""
    import numpy as np
    import torch
    import nrv_inputs as I
    from paper_2407_19097_gb300 import nrv
    dev = torch.device("cuda", 0)
    t0 = time.time()
    sc = I.terrain_scene(a.terrain_grid, seed=7)
    sizes = [(2160, 2160), (2160, 2160), (1920, 1080), (1920, 1080), (1920, 1080), (1920, 1080),
             (960, 540), (960, 540)]
    views = I.orbit_views(sc, sizes, seed=11, stereo_pairs=1)
    ds, do = I.depth_normalisation(sc, views[2])
    gen_s = time.time() - t0
    c0 = len(sc.channels) + 2
    scene = nrv.Scene(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.attr.view(np.int32)).to(dev),
                      sc.n_words)
    net = nrv.Net(c0)
    net.set_params(torch.from_numpy(unet_params(c0)).to(dev))
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    rgbs = [torch.empty((v.height, v.width, 3), dtype=torch.float32, device=dev) for v in views]
    stream = torch.cuda.current_stream()
    ms = _events_ms(lambda: nrv.render_batch(scene, net, desc, views, rgbs, nrv.PREC_BF16), a.steps,
                    a.warmup, stream)
    nrv.set_profiling(True)
    _events_ms(lambda: nrv.render_batch(scene, net, desc, views, rgbs, nrv.PREC_BF16), 5, 1, stream)
    nrv.set_profiling(False)
    st = nrv.timings()
    px = sum(v.width * v.height for v in views)
    line = {"config": "c4", "metric": "aggregate point-views/s and frames/s, 8 views",
            "workload": f"terrain {a.terrain_grid}^2 = {sc.n} points, 8 views {sizes}", "data": "synthetic",
            "value": sc.n * len(views) / (ms * 1e-3), "unit": "point-views/s",
            "frames_per_s": len(views) / (ms * 1e-3), "batch_ms": ms, "pixels_per_batch": px,
            "stages_ms": {"clear": st[0], "render_pass_all_views": st[1], "resolve_pack": st[2],
                          "network_all_views": st[3]},
            "precision": "bf16", "scene_gen_s": gen_s}
    print(json.dumps(line), flush=True)


def run_train(a):
    """The training step alone (forward, L1 loss, backward, Adam, weight repack) on seeded
    inputs of C5's shape: batch 16 of 256^2 crops, C0 = 5 (K = 3), BF16.  No targets from the
    splatter (random targets): for timing and profiling the kernels of a step."""
    import numpy as np
    import torch
    from paper_2407_19097_gb300 import nrv
    dev = torch.device("cuda", 0)
    c0, B, S = 5, 16, 256
    net = nrv.Net(c0)
    p = torch.from_numpy(unet_params(c0)).to(dev)
    net.set_params(p)
    g, m, v = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, device=dev)
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.random((B, S, S, 8), dtype=np.float32)).to(dev)
    x[..., c0:] = 0
    x = x.to(torch.bfloat16)
    t = torch.from_numpy(rng.random((B, S, S, 3), dtype=np.float32)).to(dev)
    step = [0]

    def one():
        step[0] += 1
        net.train_step(p, g, m, v, step[0], 1e-3, x, t, B, S, S, nrv.PREC_BF16, loss)

    stream = torch.cuda.current_stream()
    ms = _events_ms(one, max(a.steps, 1), max(a.warmup, 1), stream)
    line = {"config": "train", "metric": "training step time (ms)", "value": ms, "unit": "ms/step",
            "higher_is_better": False, "workload": f"batch {B} of {S}x{S}, C0={c0}, BF16",
            "pixels_per_step": B * S * S, "data": "synthetic (seeded inputs and targets)",
            "loss": float(loss.item())}
    print(json.dumps(line), flush=True)


def run_c5(a):
    """Training (Sec. 3.3) on config 3's scene (1M particles x 350 steps = 350M points): the
    U-Net learns to turn G-buffers into Gaussian-splat targets (the CPU splatter standing in for
    the paper's Gaussian Renderer), 56 training and 8 held-out hemisphere views at 512^2, random
    256^2 crops, batch 16, Adam lr 1e-3, BF16 forward/backward, 2000 steps.  Reports the step
    time; held-out PSNR/SSIM of the trained network and of the method without it (transfer-
    function colour of the winning point); the trained weights' error in BF16, FP8 and all-E4M3
    against the FP64 oracle; the same training with Eq. 1's reconstruction and TV terms; and
    the sparsity study of Tab. 6 (inputs rendered from every S-th point, targets from all)."""
    import numpy as np
    import torch
    import nrv_inputs as I
    import oracle
    from oracle import metrics, unet
    from paper_2407_19097_gb300 import nrv
    dev = torch.device("cuda", 0)
    steps = a.c5_steps
    t0 = time.time()
    full = I.trajectory_scene(a.particles, a.steps_per_particle, seed=2)
    colours = I.point_colours(full)
    size, n_views, n_train, crop, batch = 512, 64, 56, 256, 16
    views = I.hemisphere_views(full, n_views, size, size, seed=5)
    gen_s = time.time() - t0
    t0 = time.time()
    targets = [np.clip(oracle.splat(full.xyz, v, colours), 0.0, 1.0).astype(np.float32) for v in views]
    splat_s = time.time() - t0
    T = torch.from_numpy(np.stack(targets)).to(dev)
    c0 = len(full.channels) + 2
    held = range(n_train, n_views)
    stream = torch.cuda.current_stream()
    crops = [I.random_crops(9, s, batch, n_train, size, size, crop) for s in range(steps)]

    def inputs(sc, cols):
        """G-buffers of every view packed into BF16 network inputs, the colour (cols) of each
        pixel's winning point (the method without the network), a 1080p frame's time and the
        scene handle."""
        scene = nrv.Scene(torch.from_numpy(sc.xyz).to(dev), torch.from_numpy(sc.attr.view(np.int32)).to(dev),
                          sc.n_words)
        ds, do = I.depth_normalisation(full, views[0])
        desc = nrv.make_pack_desc(full.channels, ds, do)
        X, base = [], []
        for v in views:
            key = torch.empty((size, size), dtype=torch.int64, device=dev)
            x = torch.empty((size, size, 8), dtype=torch.bfloat16, device=dev)
            nrv.rasterize(scene, [v], [key])
            nrv.resolve_pack(scene, v, key, desc, nrv.PREC_BF16, x)
            X.append(x)
            k = key.cpu().numpy().view(np.uint64)
            hit = k != np.uint64(0xFFFFFFFFFFFFFFFF)
            b = np.zeros((size, size, 3), np.float32)
            b[hit] = cols[(k[hit] & np.uint64(0xFFFFFFFF)).astype(np.int64)]
            base.append(b)
        frame_ms = None
        view = I.fitted_view(full, 1920, 1080)
        net = nrv.Net(c0)
        p = torch.empty((nrv.param_count(c0),), device=dev)
        net.init_params(1, p)
        rgb = torch.empty((1080, 1920, 3), device=dev)
        frame_ms = _events_ms(lambda: nrv.render_batch(scene, net, desc, [view], [rgb], nrv.PREC_BF16),
                              20, 3, stream)
        return torch.stack(X), base, frame_ms, scene, desc

    def train(X, loss_w):
        net = nrv.Net(c0)
        p = torch.empty((nrv.param_count(c0),), device=dev)
        net.init_params(1, p)
        net.set_loss(loss_w)
        g, m, vv = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
        loss = torch.zeros(1, device=dev)
        xb = torch.empty((batch, crop, crop, 8), dtype=torch.bfloat16, device=dev)
        tb = torch.empty((batch, crop, crop, 3), dtype=torch.float32, device=dev)
        step_ms = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for s_ in range(steps):
            for b, (vi, y0, x0) in enumerate(crops[s_]):   # crops gathered outside the timed step
                xb[b].copy_(X[vi, y0:y0 + crop, x0:x0 + crop])
                tb[b].copy_(T[vi, y0:y0 + crop, x0:x0 + crop])
            if s_ >= 10:
                e0.record(stream)
            net.train_step(p, g, m, vv, s_ + 1, 1e-3, xb, tb, batch, crop, crop, nrv.PREC_BF16, loss)
            if s_ >= 10:
                e1.record(stream)
                torch.cuda.synchronize()
                step_ms.append(e0.elapsed_time(e1))
        out = torch.empty((n_views - n_train, size, size, 3), device=dev)
        net.shade(X[n_train:].contiguous(), n_views - n_train, size, size, nrv.PREC_BF16, out)
        torch.cuda.synchronize()
        return net, p, np.clip(out.cpu().numpy(), 0.0, 1.0), float(np.median(step_ms)), float(loss.item())

    def quality(imgs, base):
        return {"network_psnr_db": float(np.mean([metrics.psnr(imgs[i], targets[n_train + i]) for i in range(len(held))])),
                "network_ssim": float(np.mean([metrics.ssim(imgs[i], targets[n_train + i]) for i in range(len(held))])),
                "rasterizer_alone_psnr_db": float(np.mean([metrics.psnr(base[n_train + i], targets[n_train + i]) for i in range(len(held))])),
                "rasterizer_alone_ssim": float(np.mean([metrics.ssim(base[n_train + i], targets[n_train + i]) for i in range(len(held))]))}

    X, base, frame_ms, scene_full, desc_full = inputs(full, colours)
    net, p, imgs, step_ms, last_loss = train(X, (1.0, 0.0, 0.0))
    line = {"config": "c5", "metric": "training step time (ms) and held-out PSNR vs splat targets",
            "workload": f"trajectories {a.particles}x{a.steps_per_particle} = {full.n} points, "
                        f"{n_train}+{n_views - n_train} hemisphere views at {size}^2, {crop}^2 crops, "
                        f"batch {batch}, {steps} steps",
            "data": "synthetic", "value": step_ms, "unit": "ms/step", "higher_is_better": False,
            "precision": "bf16", "pixels_per_step": batch * crop * crop, "loss": "l1",
            "held_out": quality(imgs, base), "final_loss": last_loss,
            "scene_gen_s": gen_s, "splat_targets_s": splat_s, "cpu_cores": os.cpu_count()}
    # the trained weights in every precision against the FP64 oracle (held-out views)
    xin = X[n_train:].contiguous()
    xf = xin.float().cpu().numpy().astype(np.float64)
    flat = p.cpu().numpy()
    ref = unet.forward(xf[..., :c0], unet.unflatten(flat, c0))
    net.calibrate(X[:8].contiguous(), 8, size, size)
    inv8 = 1.0 / net.act_scales()[0]
    prec_err = {}
    for name, pr in (("bf16", nrv.PREC_BF16), ("fp8", nrv.PREC_FP8), ("fp8_e4m3", nrv.PREC_FP8_E4M3)):
        out = torch.empty((n_views - n_train, size, size, 3), device=dev)
        x_in = xin
        if pr == nrv.PREC_FP8_E4M3:
            x_in = torch.empty((n_views - n_train, size, size, 16), dtype=torch.uint8, device=dev)
            for i in range(n_views - n_train):
                key = torch.empty((size, size), dtype=torch.int64, device=dev)
                nrv.rasterize(scene_full, [views[n_train + i]], [key])
                nrv.resolve_pack(scene_full, views[n_train + i], key, desc_full, pr, x_in[i], inv8)
        net.shade(x_in, n_views - n_train, size, size, pr, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        r = float(ref.max() - ref.min())
        mse = float(np.mean((got - ref) ** 2))
        prec_err[name] = {"psnr_db": 10 * np.log10(r * r / mse) if mse > 0 else None,
                          "max_abs": float(np.abs(got - ref).max()),
                          "max_rel_to_range": float(np.abs(got - ref).max() / r)}
    line["trained_weights_vs_fp64"] = prec_err
    # Eq. 1 without its perceptual term: L2 reconstruction + total variation
    _, _, imgs2, step2, _ = train(X, (0.0, 1.0, 0.01))
    line["loss_l2_tv"] = {"weights": {"l2": 1.0, "tv": 0.01}, "step_ms": step2, **quality(imgs2, base)}
    # sparsity study (Tab. 6): inputs from every S-th point, targets from the whole scene
    sparsity = {"1": {"frame_1080p_ms": frame_ms, **line["held_out"]}}
    for S in [int(v) for v in a.sparsity.split(",") if v and int(v) > 1]:
        sel = np.arange(0, full.n, S)
        sub = full.subset(sel)
        Xs, base_s, fms, sc_s, _ = inputs(sub, colours[sel])
        _, _, imgs_s, _, _ = train(Xs, (1.0, 0.0, 0.0))
        sparsity[str(S)] = {"points": sub.n, "frame_1080p_ms": fms, **quality(imgs_s, base_s)}
        del Xs, sc_s
    line["sparsity"] = sparsity
    print(json.dumps(line), flush=True)

def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if a.config != "c3":
        import __graft_entry__
        __graft_entry__.build()
        return {"c2": run_c2, "c4": run_c4, "c5": run_c5, "train": run_train}[a.config](a)

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import nrv_inputs as I
    from paper_2407_19097_gb300 import nrv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    peaks, peak_kind = load_peaks()

    sc, view, ds, do, gen_s = make_workload(a)
    c0 = len(sc.channels) + 2
    xyz = torch.from_numpy(sc.xyz).to(dev)
    attr = torch.from_numpy(sc.attr.view(np.int32)).to(dev)
    scene = nrv.Scene(xyz, attr, sc.n_words)
    net = nrv.Net(c0)
    params = torch.from_numpy(unet_params(c0)).to(dev)
    net.set_params(params)
    desc = nrv.make_pack_desc(sc.channels, ds, do)
    H, W = view.height, view.width
    rgb = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    prec = nrv.PREC_BF16 if a.prec == "bf16" else nrv.PREC_F32
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(prec_, steps, warmup, profile, inv=1.0):
        for _ in range(warmup):
            nrv.render_batch(scene, net, desc, [view], [rgb], prec_, inv)
        torch.cuda.synchronize()
        nrv.timings()
        nrv.set_profiling(profile)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = nrv.lib().nrv_launch_count()
        e0.record(stream)
        for _ in range(steps):
            nrv.render_batch(scene, net, desc, [view], [rgb], prec_, inv)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = nrv.lib().nrv_launch_count() - n0
        barrier()
        nrv.set_profiling(False)
        stages = nrv.timings() if profile else None
        return e0.elapsed_time(e1) / steps, stages, launches

    # the timed step: whole frames as a user runs them (captured once, replayed)
    sampler = ClockSampler(local)
    sampler.start()
    ms, _, launches = timed(prec, a.steps, a.warmup, False)
    clocks = sampler.stop()
    # stage times: the same frames run eagerly with events between the stages
    _, stages, _ = timed(prec, max(5, a.steps // 5), 2, True)
    # the render pass without chunk culling (the variant every point goes through)
    pinned = os.environ.get("NRV_VIS_VARIANT")
    os.environ["NRV_VIS_VARIANT"] = "0"
    _, stages_bf, _ = timed(prec, max(5, a.steps // 5), 2, True)
    if pinned is None:
        del os.environ["NRV_VIS_VARIANT"]
    else:
        os.environ["NRV_VIS_VARIANT"] = pinned
    ms, value = job_rate(ms, sc.n, world, dev)

    # end to end through the public API: camera from the host, every frame back to pinned host
    # memory.  Frames alternate between two output buffers; frame i's copy runs on a copy
    # stream while frame i + 1 renders, and the host waits for frame i's copy (and reads a
    # pixel of it) before it submits frame i + 2.
    rgbs = [rgb, torch.empty_like(rgb)]
    hosts = [torch.empty((H, W, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    copy_stream = torch.cuda.Stream()

    def e2e_frames(k):
        copied = [None, None]
        check = 0.0
        for i in range(k):
            b = i % 2
            if copied[b] is not None:
                copied[b].synchronize()               # frame i - 2 is on the host
                check += float(hosts[b][0, 0, 0])
                stream.wait_event(copied[b])          # its buffer may be overwritten
            nrv.render_batch(scene, net, desc, [view], [rgbs[b]], prec)
            rendered = torch.cuda.Event()
            rendered.record(stream)
            copy_stream.wait_event(rendered)
            with torch.cuda.stream(copy_stream):
                hosts[b].copy_(rgbs[b], non_blocking=True)
                copied[b] = torch.cuda.Event()
                copied[b].record(copy_stream)
        for b in range(2):
            if copied[b] is not None:
                copied[b].synchronize()
                check += float(hosts[b][0, 0, 0])
        return check

    e2e_frames(max(a.warmup, 2))
    barrier()
    t0 = time.perf_counter()
    e2e_frames(a.steps)
    e2e_s = (time.perf_counter() - t0) / a.steps
    barrier()

    local_peaks = measure_local_peaks(dev) if rank == 0 else None

    # the FP32 form of the same pipeline, for comparison
    fp32_ms = None
    if not a.no_fp32 and prec != nrv.PREC_F32:
        fp32_ms, _, _ = timed(nrv.PREC_F32, max(3, a.steps // 10), 2, False)

    # the FP8 networks, calibrated on this frame's BF16 input: NRV_PREC_FP8 (E4M3 levels 1-3,
    # BF16 level 0) and NRV_PREC_FP8_E4M3 (every tensor E4M3, below the accuracy bar)
    fp8_ms, fp8_rgb, e4m3_ms, e4m3_rgb = None, None, None, None
    if not a.no_fp8:
        key = torch.empty((H, W), dtype=torch.int64, device=dev)
        dpl = torch.empty((H, W), dtype=torch.int32, device=dev)
        msk = torch.empty((H, W), dtype=torch.uint8, device=dev)
        gat = torch.empty((sc.n_words, H, W), dtype=torch.int32, device=dev)
        nrv.rasterize(scene, [view], [key], [dpl], [msk], [gat])
        xb = torch.empty(((H + 7) // 8 * 8, (W + 7) // 8 * 8, 8), dtype=torch.bfloat16, device=dev)
        nrv.pack(dpl, msk, gat, H, W, desc, nrv.PREC_BF16, xb)
        net.calibrate(xb, 1, H, W)
        inv8 = 1.0 / net.act_scales()[0]
        del key, dpl, msk, gat, xb
        fp8_ms, _, _ = timed(nrv.PREC_FP8, max(5, a.steps // 5), 3, False)
        nrv.render_batch(scene, net, desc, [view], [rgb], nrv.PREC_FP8)
        torch.cuda.synchronize()
        fp8_rgb = rgb.float().cpu().numpy().astype(np.float64)
        e4m3_ms, _, _ = timed(nrv.PREC_FP8_E4M3, max(5, a.steps // 5), 3, False, inv8)
        nrv.render_batch(scene, net, desc, [view], [rgb], nrv.PREC_FP8_E4M3, inv8)
        torch.cuda.synchronize()
        e4m3_rgb = rgb.float().cpu().numpy().astype(np.float64)

    # the gated network (Sec. 3.3's form) on this frame's BF16 input: time and tensor fraction
    gated_line = None
    if not a.no_gated:
        key = torch.empty((H, W), dtype=torch.int64, device=dev)
        nrv.rasterize(scene, [view], [key])
        xb = torch.empty(((H + 7) // 8 * 8, (W + 7) // 8 * 8, 8), dtype=torch.bfloat16, device=dev)
        nrv.resolve_pack(scene, view, key, desc, nrv.PREC_BF16, xb)
        gnet = nrv.GatedNet(c0)
        gnet.set_params(torch.from_numpy(gated_params(c0)).to(dev))
        grgb = torch.empty((H, W, 3), device=dev)
        g_ms = _events_ms(lambda: gnet.shade(xb, 1, H, W, grgb), max(10, a.steps // 5), 3, stream)
        gfl = gated_flops_per_frame(H, W, c0)
        pk_t = peaks.get("bf16_tflops_sustained", 1700.0)
        gated_line = {"ms": g_ms, "flops_per_frame": gfl, "achieved_tflops": gfl / (g_ms * 1e-3) / 1e12,
                      "tensor_peak_tflops": pk_t, "frac": gfl / (g_ms * 1e-3) / 1e12 / pk_t,
                      "widths": "16/32/64/128 (gated: feature + gate)"}
        del key, xb, gnet

    # roofline of the render pass (the dominant stage).  The culling pass reads every chunk box
    # but the positions only of the points it cannot rule out: its algorithmic bytes are those
    # reads (data-dependent; measured with ncu for the default workload), not 12 B for every
    # point -- that figure over the same time is reported as effective_gbs
    clear_ms, vis_ms, res_ms, net_ms = stages
    vis_gbs = sc.n * BYTES_PER_POINT / (vis_ms * 1e-3) / 1e9
    bf_ms = stages_bf[1]
    bf_gbs = sc.n * BYTES_PER_POINT / (bf_ms * 1e-3) / 1e9
    known = (a.particles, a.steps_per_particle, W, H) == (1_000_000, 350, 1920, 1080)
    moved_gbs = RENDER_TRAFFIC_BYTES / (vis_ms * 1e-3) / 1e9 if known else vis_gbs
    roof = {"kernel": "render pass (chunk_render_kernel x3 + tile_bound_kernel x2 + "
                      "tile_pyramid_kernel x2, tuned variant)",
            "bound": "hbm", "achieved": moved_gbs,
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": moved_gbs / peaks["hbm_gbs"],
            "traffic": RENDER_TRAFFIC_BYTES if known else None,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum summed over the "
                              "render pass's seven launches of one frame (variant "
                              "single/chunks/16x2/r/sub/hiz/33), "
                              "profiles/render_pass_dram_traffic_trajectories_350m_1080p.md",
            "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": RENDER_TRAFFIC_BYTES if known else sc.n * BYTES_PER_POINT,
            "algorithmic_bytes_definition": (
                "the reads the culling pass cannot avoid on this frame: every 32-point chunk box, "
                "the sub-chunk boxes of surviving chunks, the positions of the prepass chunks and "
                "of the surviving sub-chunks, plus tile bounds and atomics (measured)" if known else
                "12 B per point (no capture of this workload: an effective figure)"),
            "effective_gbs": vis_gbs,
            "note": "the pass is bound by instruction issue and memory latency (box tests, exact "
                    "projection, one early depth read per projected point), not by DRAM: it runs "
                    "far below the HBM roofline of the bytes it moves; effective_gbs is 12 B per "
                    "point over the same time, the rate a pass reading every point would need"}
    roof_bf = {"kernel": "visibility_kernel (brute force, every point)", "bound": "hbm",
               "achieved": bf_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
               "frac": bf_gbs / peaks["hbm_gbs"], "ms": bf_ms, "peak_source": peak_kind}
    flops = 71424.0 * (H + (-H) % 8) * (W + (-W) % 8)
    net_tf = flops / (net_ms * 1e-3) / 1e12
    pk = peaks.get("bf16_tflops_sustained", 1700.0)
    net_floor = network_floor_ms(H, W, c0, peaks["hbm_gbs"], pk)

    line = {"metric": "points/s (frames/s) at 1080p", "value": value, "unit": "points/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "fps": 1e3 / ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": a.prec, "data": "synthetic",
            "config": {"workload": workload_name(a), "network": f"U-Net 16/32/64/128, C_in={c0}",
                       "precision": a.prec, "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"inputs larger than L2 ({sc.n * BYTES_PER_POINT / 1e9:.2f} GB of "
                             f"point positions per frame)"},
            "stages_ms": {"clear": clear_ms, "visibility": vis_ms, "resolve_pack": res_ms,
                          "network": net_ms},
            "roofline": roof,
            "roofline_render_brute_force": roof_bf,
            "roofline_network": {"bound": "tensor", "achieved": net_tf, "peak": pk,
                                 "unit": "TFLOP/s", "frac": net_tf / pk,
                                 "flops_per_frame": flops,
                                 "stage_floor_ms": net_floor,
                                 "frac_of_stage_floor": net_floor / net_ms,
                                 "stage_floor_note": "sum over layers of max(FLOP time at the "
                                 "sustained tensor peak, byte time at the HBM peak)"},
            "fp32_ms_per_step": fp32_ms,
            "local_peaks": local_peaks,
            "roofline_network_fp32": (
                {"bound": "alu", "achieved": flops / ((fp32_ms - clear_ms - vis_ms - res_ms) * 1e-3) / 1e12,
                 "peak": local_peaks["fp32_ffma_tflops"], "unit": "TFLOP/s",
                 "frac": flops / ((fp32_ms - clear_ms - vis_ms - res_ms) * 1e-3) / 1e12
                 / local_peaks["fp32_ffma_tflops"],
                 "note": "FP32 network (CUDA cores) time = FP32 frame minus the BF16 frame's "
                         "clear, render and resolve stages; peak from the FFMA probe"}
                if fp32_ms and local_peaks else None),
            "gated_network": gated_line,
            "fp8_ms_per_step": fp8_ms,
            "fp8_e4m3_ms_per_step": e4m3_ms,
            "e2e": {"value": world * sc.n / e2e_s, "unit": "points/s",
                    "h2d_bytes_per_step": VIEW_TABLE_BYTES, "d2h_bytes_per_step": H * W * 3 * 4,
                    "copies": "each frame's RGB copy to pinned host memory overlaps the next "
                              "frame's render (two output buffers, a copy stream)"},
            "clocks": clocks, "scene_gen_s": gen_s}
    # library kernels launched inside the timed region (counted by the library)
    line["gpu_launches"] = int(launches)

    if rank == 0 and not a.no_cpu_baseline:
        nrv.render_batch(scene, net, desc, [view], [rgb], prec)
        torch.cuda.synchronize()
        t_cpu, y_ref, t_ras = oracle_frame(sc, view, ds, do)
        # the oracle's render pass on all cores, and its splatter (the GR stand-in) on one view
        import oracle as _oracle
        t0 = time.perf_counter()
        _oracle.visibility(sc.xyz, view, threads="all")
        t_ras_all = time.perf_counter() - t0
        sview = I.hemisphere_views(sc, 1, 512, 512, seed=5)[0]
        cols = I.point_colours(sc)
        t0 = time.perf_counter()
        _oracle.splat(sc.xyz, sview, cols)
        t_splat = time.perf_counter() - t0
        got = rgb.float().cpu().numpy().astype(np.float64)
        r = float(y_ref.max() - y_ref.min())
        mse = float(np.mean((got - y_ref) ** 2))
        line["cpu_baseline"] = {"value": sc.n / t_cpu, "unit": "points/s", "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": "one whole frame: render+resolve+pack in C on one thread "
                                          f"({t_ras:.1f} s), FP64 U-Net in numpy on all BLAS "
                                          f"threads ({t_cpu - t_ras:.1f} s)",
                                "render_pass_points_per_s": {"one_thread": sc.n / t_ras,
                                                             "all_cores": sc.n / t_ras_all},
                                "splat_target_s_per_view_512": t_splat}
        line["quality_vs_fp64"] = {"psnr_db": 10 * np.log10(r * r / mse) if mse > 0 else None,
                                   "max_abs": float(np.abs(got - y_ref).max())}
        for key8, img in (("quality_fp8_vs_fp64", fp8_rgb), ("quality_fp8_e4m3_vs_fp64", e4m3_rgb)):
            if img is not None:
                mse8 = float(np.mean((img - y_ref) ** 2))
                line[key8] = {"psnr_db": 10 * np.log10(r * r / mse8) if mse8 > 0 else None,
                              "max_abs": float(np.abs(img - y_ref).max())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
