#!/usr/bin/env python
"""Benchmark: 1080p multi-scale TTC/FOE frame pairs per second on GB300.

One step = the whole hot path over one synthetic video: 300 uint8 1920x1080 frames
of a textured plane tilted 20 degrees (camera within 15 degrees of the optical axis,
Z0 = 20, 0.05 per frame), 5-level pyramid, 2x2x2 derivatives, G, the ten sums, FP64
merge and 3x3 FOE solve for all 299 consecutive pairs: one streaming pass per level
(level 0 by the persistent TMA-fed kernel, levels 1-4 by interior and edge launches
of the pass kernel, each writing the next level) and one merge/solve launch.  The
622 MB video is larger than L2 (129 MB), so no flush is needed between steps.

Also reported in the same JSON line:
  roofline       of the level-0 pass (CUDA events on its stream inside the timed
                 region): FP32 lane-ops per second against the FP32 issue roof, with
                 its HBM rate beside it
  e2e            the same metric through the public API with pinned host frames
                 (H2D copy of the video and D2H of the results inside the timed region)
  cpu_baseline   the FP64 oracle on a bounded sample of the same video, one core
  fastconv       the FastConv sweep (1080x1920 with k x k Gaussians, 64x256x256 with
                 k^3, batches of 16 images) in GB/s and GFLOP/s with the fraction of
                 the HBM or FP32 FMA roof, L2 flushed between runs; separable Gaussians
                 through one 1-D pass per axis against the direct path
  gradient       gradient magnitude and direction of 1080p uint8 images, GB/s
  batch_uneven   512 independent pairs of uneven sizes in one batch (the all-levels
                 kernel and the merge/solve, replayed from a CUDA graph) against the
                 per-frame path, with every pair's error against the FP64 oracle
  serve          64 camera streams replayed at 30 fps through the serving loop and
                 through the per-frame path (p50/p99 latency), then saturated
  accuracy       TTC/FOE mean squared error against ground truth per level and per
                 multi-scale rule (Sec. V-B)
  clocks         nvidia-smi samples taken during the timed region

``--impl reference`` times the FP64 oracle (the only reference that exists for this
method) on a bounded sample of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "1080p multi-scale TTC frame-pairs/s; conv HBM GB/s % of peak; serve p50/p99 ms"
UNIT = "frame-pairs/s"
H, W, T_FRAMES, LEVELS = 1080, 1920, 300, 5
# sum tolerance for uint8 frames, relative to the oracle's error scale (57 roundings of
# 2^-24 on any term's path: see the parity tests' tolerance module)
SUM_TOL_U8 = 3.5e-6
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def _config(frames):
    return {"workload": f"ttc_video_1080p_{frames}frames_{LEVELS}levels_foe",
            "H": H, "W": W, "frames": frames, "pairs_per_step": frames - 1, "levels": LEVELS,
            "mode": "foe", "frame_dtype": "u8",
            "l2": "inputs 622 MB per step > 129 MB L2 (no flush needed)"}


# --------------------------------------------------------------------------- #
# clocks
# --------------------------------------------------------------------------- #

def _smi_index(local: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local < len(ids):
            return ids[local]
    return str(local)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.proc = None
        self.idx = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- #
# reference arm: the FP64 oracle on the host
# --------------------------------------------------------------------------- #

def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return 0
    import oracle
    import scenes
    oracle.build()
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=args.seed)
    pairs_per_step = args.ref_pairs
    fr = scenes.render_sequence(sc, pairs_per_step + 1).numpy()
    for _ in range(args.warmup):
        oracle.ttc_pair(fr[0], fr[1], levels=LEVELS, mode=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for t in range(pairs_per_step):
            oracle.ttc_pair(fr[t], fr[t + 1], levels=LEVELS, mode=1)
    dt = time.perf_counter() - t0
    value = pairs_per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(_config(T_FRAMES), sample=f"{pairs_per_step} pairs of the video per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{pairs_per_step} 1080p pairs x {args.steps} steps, 5 levels, FOE",
                         "nproc": host_cpu()["nproc"], "cpu_model": host_cpu()["model"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #

class L2Flush:
    """Between timed launches: write a buffer larger than L2 (evicts the launch's inputs),
    then read another one as large, so that the dirty lines of the write are written back
    before the timed launch rather than during it; L2 is left holding clean lines of
    neither the inputs nor the outputs.  Then the device spins for about 0.3 ms, so that
    the host has enqueued the timed call before the device reaches the call's start event:
    the events then time the device's work, not the host-side marshalling of a short call
    (which the small-call measurements report separately)."""

    SPIN_CYCLES = 600_000

    def __init__(self, dev):
        import torch
        self.torch = torch
        self.w = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.zero_()
        self.r.sum()
        self.torch.cuda._sleep(self.SPIN_CYCLES)


def single_launch_us(dev, flush, fn, reps):
    """Median device time of one call between CUDA events, L2 flushed before each."""
    import torch
    s = torch.cuda.current_stream(dev)
    times = []
    for _ in range(reps + 2):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        times.append((e0, e1))
    torch.cuda.synchronize(dev)
    return float(np.median([a.elapsed_time(b) for a, b in times[2:]])) * 1e3


def fastconv_sweep(dev, hbm_peak, fma_peak, reps):
    import torch
    import paper_1612_08825_gb300 as ft
    import scenes
    flush = L2Flush(dev)
    rows = []
    # the sweep's shapes, plus batches of 16 images (a leading extent-1 kernel axis)
    # that show the sustained rates: a single 1080p image is too small to fill the GPU
    cases = [((1080, 1920), (k, k), "gauss") for k in (2, 3, 7, 15)] + \
            [((64, 256, 256), (k, k, k), "normal") for k in (2, 5)] + \
            [((16, 1080, 1920), (1, k, k), "gauss") for k in (2, 3, 5, 7, 15)]
    launches = 0
    for shape, kshape, kind in cases:
        E = torch.from_numpy(scenes.uniform_array(shape, seed=2024)).to(dev)
        if kind == "gauss":
            k = torch.from_numpy(scenes.gaussian_kernel(kshape[-1]).reshape(kshape)).to(dev)
        else:
            k = torch.from_numpy(scenes.normal_array(kshape, seed=78)).to(dev)
        out = ft.fastconv_nd(E, k)
        s = torch.cuda.current_stream(dev)
        times = []
        for i in range(reps + 2):
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ft.fastconv_nd(E, k, out=out)
            e1.record(s)
            launches += 1
            times.append((e0, e1))
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(b) for a, b in times[2:]]
        t = float(np.median(ms)) * 1e-3
        nE, nk, no = E.numel(), k.numel(), out.numel()
        byts = 4 * (nE + no + nk)
        flops = 2.0 * nE * nk
        gbs = byts / t / 1e9
        bound = "fma" if flops / byts > fma_peak / (hbm_peak * 1e9) else "hbm"
        row = {"input": list(shape), "kernel": list(kshape), "us": t * 1e6, "bound": bound,
               "GBps": gbs, "hbm_frac": gbs / hbm_peak, "GFLOPps": flops / t / 1e9,
               "fma_frac": flops / t / fma_peak, "algorithmic_bytes": byts, "flops": flops}
        if bound == "hbm":
            # the same single-launch timing of a device copy of the same bytes (read the
            # input, write as many bytes): what one launch of this size can reach here
            dst = torch.empty(max(no, nE), dtype=torch.float32, device=dev)
            row["copy_same_bytes_us"] = single_launch_us(
                dev, flush, lambda: dst[:nE].copy_(E.reshape(-1)), reps) if no >= nE else None
            if row["copy_same_bytes_us"]:
                row["frac_of_copy"] = row["copy_same_bytes_us"] / row["us"]
        rows.append(row)
    # inputs of other element types, staged by the copy engine in their own type and
    # widened in the kernel: bytes = input bytes + FP32 output
    for shape, kshape, dt in (((16, 1080, 1920), (1, 3, 3), torch.uint8), ((16, 1080, 1920), (1, 7, 7), torch.uint8),
                              ((16, 1080, 1920), (1, 5, 5), torch.float16)):
        Ef = torch.from_numpy(scenes.uniform_array(shape, seed=2024)).to(dev)
        E = (Ef * 255).to(torch.uint8) if dt == torch.uint8 else Ef.to(dt)
        k = torch.from_numpy(scenes.gaussian_kernel(kshape[-1]).reshape(kshape)).to(dev)
        out = ft.fastconv_nd(E, k)
        ts = []
        for i in range(reps + 2):
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ft.fastconv_nd(E, k, out=out)
            e1.record(s)
            ts.append((e0, e1))
        torch.cuda.synchronize(dev)
        launches += reps + 2
        t = float(np.median([a.elapsed_time(b) for a, b in ts[2:]])) * 1e-3
        byts = E.numel() * E.element_size() + 4 * (out.numel() + k.numel())
        flops = 2.0 * E.numel() * k.numel()
        bound = "fma" if flops / byts > fma_peak / (hbm_peak * 1e9) else "hbm"
        rows.append({"input": list(shape), "kernel": list(kshape), "input_dtype": str(dt).replace("torch.", ""),
                     "us": t * 1e6, "bound": bound, "GBps": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / hbm_peak,
                     "GFLOPps": flops / t / 1e9, "fma_frac": flops / t / fma_peak, "algorithmic_bytes": byts,
                     "flops": flops})

    # direct vs FFT on one 1080 x 1920 image with K x K N(0,1) kernels: where the FFT
    # path starts to win (the paper's switch, Sec. IV-D)
    Ec = torch.from_numpy(scenes.uniform_array((1080, 1920), seed=2024)).to(dev)
    cross = []
    for K in (9, 15, 21, 25, 31, 41, 51, 63):
        k = torch.from_numpy(scenes.normal_array((K, K), seed=K)).to(dev)
        out = ft.fastconv_nd(Ec, k)
        plan = ft.FftPlan(tuple(Ec.shape), (K, K), dev)
        ws = plan.new_workspace()
        t_dir, t_fft = [], []
        for i in range(reps + 2):
            for fn, acc in ((lambda: ft.fastconv_nd(Ec, k, out=out), t_dir),
                            (lambda: plan(Ec, k, out=out, workspace=ws), t_fft)):
                flush()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                fn()
                e1.record(s)
                acc.append((e0, e1))
        torch.cuda.synchronize(dev)
        td = float(np.median([a.elapsed_time(b) for a, b in t_dir[2:]])) * 1e3
        tf = float(np.median([a.elapsed_time(b) for a, b in t_fft[2:]])) * 1e3
        cross.append({"K": K, "direct_us": td, "fft_us": tf, "faster": "fft" if tf < td else "direct"})
    import ctypes
    L = ft.load()
    auto = [K for K in range(3, 80) if L.fastconv_prefers_fft((ctypes.c_int64 * 2)(1080, 1920), 2,
                                                              (ctypes.c_int64 * 2)(K, K))]
    rows.append({"input": [1080, 1920], "crossover_direct_vs_fft": cross,
                 "library_switches_to_fft_at_K": auto[0] if auto else None})

    # separable kernels through one 1-D pass per axis (normalised Gaussians): time and
    # the speedup over the direct path for the same output
    def timed(fn):
        ts = []
        for i in range(reps + 2):
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            ts.append((e0, e1))
        torch.cuda.synchronize(dev)
        return float(np.median([a.elapsed_time(b) for a, b in ts[2:]])) * 1e-3

    for shape, ksz in (((1080, 1920), 15), ((16, 1080, 1920), 15), ((64, 256, 256), 5)):
        E = torch.from_numpy(scenes.uniform_array(shape, seed=2024)).to(dev)
        g = scenes.gaussian_kernel(ksz, ndim=1)
        nsep = 2 if len(shape) == 3 and shape[0] == 16 else len(shape)
        ks = [1] * (len(shape) - nsep) + [ksz] * nsep
        facs = [torch.ones(1, device=dev)] * (len(shape) - nsep) + [torch.from_numpy(g).to(dev)] * nsep
        full = facs[0].cpu().numpy().astype(np.float64)
        for f in facs[1:]:
            full = np.multiply.outer(full, f.cpu().numpy().astype(np.float64))
        kfull = torch.from_numpy(full.astype(np.float32)).to(dev)
        out = ft.fastconv_nd(E, kfull)
        scratch = torch.empty_like(out)
        t_sep = timed(lambda: ft.fastconv_separable(E, facs, out=out, scratch=scratch))
        t_dir = timed(lambda: ft.fastconv_nd(E, kfull, out=out))
        launches += 2 * (reps + 2) * (1 + len(shape))
        flops = 2.0 * E.numel() * kfull.numel()
        cur, byts = list(shape), 0
        for d, k in enumerate(ks):          # every pass reads its input and writes its output
            nxt = list(cur)
            nxt[d] += k - 1
            byts += 4 * (int(np.prod(cur)) + int(np.prod(nxt)))
            cur = nxt
        rows.append({"input": list(shape), "kernel": ks, "path": "separable", "us": t_sep * 1e6,
                     "bound": "hbm", "GBps": byts / t_sep / 1e9, "hbm_frac": byts / t_sep / 1e9 / hbm_peak,
                     "algorithmic_bytes": byts, "direct_us": t_dir * 1e6, "speedup_vs_direct": t_dir / t_sep,
                     "direct_equivalent_GFLOPps": flops / t_sep / 1e9})
    # the device-side cost of one launch under this timing (a 1-element convolution)
    one = torch.ones(1, device=dev)
    o1 = ft.fastconv_nd(one, one)
    rows.append({"single_launch_floor_us": single_launch_us(dev, flush, lambda: ft.fastconv_nd(one, one, out=o1),
                                                            reps),
                 "note": "a 1-element convolution timed like the rows above (L2 flush, device spin, "
                         "events): the floor of any single launch"})
    del flush
    return rows, launches


def gradient_bench(dev, hbm_peak, reps):
    """Gradient magnitude and direction (Sec. II) of one 1080p uint8 image and of 16
    images (one launch per image, and one batched launch): bytes = pixels read once +
    two float outputs written."""
    import torch
    import paper_1612_08825_gb300 as ft
    import scenes
    flush = L2Flush(dev)
    rows = []
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=5)
    img = scenes.render(sc, 0.0, device=dev)
    s = torch.cuda.current_stream(dev)
    L = ft.load()
    for n, batched in ((1, False), (16, False), (16, True)):
        stack = img.unsqueeze(0).repeat(n, 1, 1).contiguous()
        mags = torch.empty((n, H - 1, W - 1), device=dev)
        angs = torch.empty((n, H - 1, W - 1), device=dev)
        ts = []
        for i in range(reps + 2):
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            if batched:      # one launch for the batch
                L.ttc_gradient_batch(stack.data_ptr(), n, H * W, 0, H, W, W, mags.data_ptr(), angs.data_ptr(),
                                     s.cuda_stream)
            else:            # one launch per image
                for k in range(n):
                    L.ttc_gradient(stack[k].data_ptr(), 0, H, W, W, mags[k].data_ptr(), angs[k].data_ptr(),
                                   s.cuda_stream)
            e1.record(s)
            ts.append((e0, e1))
        torch.cuda.synchronize(dev)
        t = float(np.median([a.elapsed_time(b) for a, b in ts[2:]])) * 1e-3
        byts = n * (H * W + 8 * (H - 1) * (W - 1))
        rows.append({"images": n, "launches": 1 if batched or n == 1 else n, "H": H, "W": W, "dtype": "u8",
                     "us": t * 1e6, "GBps": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / hbm_peak,
                     "algorithmic_bytes": byts})
    del flush
    return rows


def small_bench(dev, reps=50):
    """The plain single-scale case: 32 float32 frames of 128 x 128 (a fronto-parallel plane
    approaching at W = 0.1 per frame from Z0 = 10), all 31 pairs in one call, TTC-only
    (C = -sum(G Et) / sum(G^2)) and FOE; and one 128 x 128 (*) 3 x 3 N(0,1) full
    convolution.  Too small for a roofline: latency per call as a caller sees it (CUDA
    events around the Python call, so the host-side marshalling gap before the launch,
    during which the GPU waits, is included) and per pair."""
    import torch
    import paper_1612_08825_gb300 as ft
    import scenes
    sc = scenes.fronto_parallel_scene(H=128, W=128, seed=0, Z0=10.0, speed=0.1)
    fr = scenes.render_sequence(sc, 32, device=dev)
    ctx = ft.TtcContext(128, 128, 1, 31, device=dev)
    out = ctx.new_results(31)
    s = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            ts.append((e0, e1))
        torch.cuda.synchronize(dev)
        return float(np.median([a.elapsed_time(b) for a, b in ts])) * 1e3

    row = {"workload": "32 float32 frames 128 x 128, 31 pairs per call, 1 level",
           "timing": "CUDA events around the Python call (includes the launch gap)"}
    for name, mode in (("ttc_only", ft.MODE_TTC), ("foe", ft.MODE_FOE)):
        us = timed(lambda: ctx.solve_sequence(fr, levels=1, mode=mode, out=out))
        row[name] = {"us_per_call": us, "us_per_pair": us / 31}
    ctx.close()
    x = torch.from_numpy(scenes.uniform_array((128, 128), seed=1)).to(dev)
    k = torch.from_numpy(scenes.normal_array((3, 3), seed=2)).to(dev)
    y = ft.fastconv_nd(x, k)
    row["conv_128x128_3x3_us"] = timed(lambda: ft.fastconv_nd(x, k, out=y))
    return row


def batch_bench(dev, args):
    """512 independent pairs of uneven sizes: autotuned work-list launches replayed from
    a CUDA graph, against the plain per-frame path (one ttc_solve per pair)."""
    import torch
    import paper_1612_08825_gb300 as ft
    import scenes
    n = args.batch_pairs
    specs = scenes.uneven_pair_sizes(n, seed=args.seed + 77)
    pairs = []
    for i, (h, w, z0, sp) in enumerate(specs):
        sc = scenes.tilted_plane_scene(H=h, W=w, seed=args.seed + 1000 + i, Z0=z0, speed=sp)
        fr = scenes.render_sequence(sc, 2, device=dev)
        # frame buffers with row pitch rounded up to 64 bytes (as camera and decoder
        # surfaces are laid out); the frames are the W-pixel views of those rows
        buf = torch.zeros((2, h, -(-w // 64) * 64), dtype=torch.uint8, device=dev)
        buf[:, :, :w] = fr
        pairs.append((buf[0, :, :w], buf[1, :, :w]))
    px = sum(h * w for h, w, _, _ in specs)
    cubes = sum(((h >> l) - 1) * ((w >> l) - 1) for h, w, _, _ in specs for l in range(LEVELS))
    ctx = ft.TtcContext(1080, 1920, LEVELS, n, device=dev)
    ctx.batch_prepare(pairs, levels=LEVELS)
    out = ctx.new_results(n * LEVELS)
    rows = ctx.batch_autotune(mode=ft.MODE_FOE, reps=2, out=out)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        ctx.batch_run(mode=ft.MODE_FOE, out=out)
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ctx.batch_run(mode=ft.MODE_FOE, out=out)
    launches = ctx.last_launch_count
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.batch_steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    t_graph = e0.elapsed_time(e1) * 1e-3 / args.batch_steps
    res = ft.results_to_numpy(out).reshape(n, LEVELS)
    # the plain per-frame path on the same GPU
    single = ft.TtcContext(1080, 1920, LEVELS, 1, device=dev)
    souts = [single.new_results(LEVELS) for _ in range(n)]
    for i, (a, b) in enumerate(pairs[:8]):
        single.solve(a, b, levels=LEVELS, mode=ft.MODE_FOE, out=souts[i])
    torch.cuda.synchronize(dev)
    e0.record()
    for i, (a, b) in enumerate(pairs):
        single.solve(a, b, levels=LEVELS, mode=ft.MODE_FOE, out=souts[i])
    e1.record()
    torch.cuda.synchronize(dev)
    t_single = e0.elapsed_time(e1) * 1e-3
    sres = np.concatenate([ft.results_to_numpy(o) for o in souts]).reshape(n, LEVELS)
    # norm-wise relative difference of the ten sums per (pair, level)
    agree = float(np.max(np.abs(sres["sums"] - res["sums"]).max(axis=-1) /
                         np.maximum(np.abs(sres["sums"]).max(axis=-1), 1e-300)))
    ctx.close()
    single.close()
    oracle_err = None
    if not args.no_batch_oracle:
        oracle_err = batch_oracle_errors(pairs, res, LEVELS)
    return {"workload": f"{n} independent uint8 pairs, W 160-1920, H 120-1080, {LEVELS} levels, FOE, "
                        "rows pitched to 64 bytes",
            "megapixels_per_frame_set": px / 1e6, "rows_per_tile_per_level": rows,
            "launches_per_batch": launches, "cubes_per_batch": cubes,
            "cubes_per_s": cubes / t_graph,
            "fp32_issue_frac": cubes * OPS_PER_CUBE0 / t_graph / alu_roof(dev),
            "graph_pairs_per_s": n / t_graph, "graph_ms_per_batch": t_graph * 1e3,
            "per_frame_path_pairs_per_s": n / t_single, "per_frame_path_ms": t_single * 1e3,
            "speedup_vs_per_frame_path": t_single / t_graph,
            "max_rel_sum_diff_vs_per_frame_path": agree,
            "vs_oracle": oracle_err}


def batch_oracle_errors(pairs, res, levels):
    """Error of every record of the batch against the FP64 oracle (all pairs, all
    levels), the oracle spread over the host cores: per pair the worst sum error
    (|got - ref| / abssum over the ten sums and all levels), and over the batch the
    worst relative TTC error and the worst FOE error in level-0 pixels."""
    import oracle
    host = [(a.cpu().numpy(), b.cpu().numpy()) for a, b in pairs]
    refs, secs = oracle.ttc_pairs_list(host, levels, 1, os.cpu_count() or 1)
    per_pair, ttc_rel, foe_px, flags_equal = [], 0.0, 0.0, True
    for i, ref in enumerate(refs):
        worst = 0.0
        for l in range(levels):
            g, r = res[i, l], ref[l]
            worst = max(worst, float(np.max(np.abs(g["sums"] - r["sums"]) / np.maximum(r["abssums"], 1e-300))))
            flags_equal &= int(g["flags"]) == int(r["flags"])
            if int(r["flags"]) & 1 or not np.isfinite(r["ttc"]):
                continue
            ttc_rel = max(ttc_rel, abs(float(g["ttc"]) - float(r["ttc"])) / abs(float(r["ttc"])))
            foe_px = max(foe_px, abs(float(g["x0"]) - float(r["x0"])), abs(float(g["y0"]) - float(r["y0"])))
        per_pair.append(worst)
    return {"pairs": len(refs), "levels": levels, "oracle_seconds": secs,
            "max_sum_err_rel_abssum": max(per_pair), "median_sum_err_rel_abssum": float(np.median(per_pair)),
            "sum_tolerance": SUM_TOL_U8, "within_sum_tolerance": int(sum(e <= SUM_TOL_U8 for e in per_pair)),
            "max_ttc_rel_err": ttc_rel, "max_foe_err_px": foe_px, "flags_identical": bool(flags_equal),
            "per_pair_max_sum_err": [float(f"{e:.3g}") for e in per_pair]}


def h2d_link_gbs(dev, nbytes, reps=5):
    """Host-to-device rate of one copy of nbytes from page-locked memory (median of reps)."""
    import torch
    src = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dst = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(reps + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record()
        dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize(dev)
        ts.append(e0.elapsed_time(e1) * 1e-3)
    return nbytes / statistics.median(ts[1:]) / 1e9


def serve_bench(dev, args):
    """Serving: 64 camera streams (16 each of 320x240, 640x480, 1280x720, 1920x1080),
    uint8, 4 levels, FOE; Poisson arrivals at 30 fps per stream replayed in real time
    through the continuous-batching server and through the plain per-frame path, then
    both saturated; plus admission under a small HBM budget."""
    import torch
    import scenes
    from paper_1612_08825_gb300.serve import (CudaBatchEngine, NativeServer, PerFrameEngine, Server,
                                              latency_summary, replay, saturate)
    levels, K = 4, 4
    specs = scenes.camera_streams(16, seed=args.seed)
    frames = {}
    for sid, H, W, seed, Z0, sp in specs:
        sc = scenes.tilted_plane_scene(H, W, seed=seed, Z0=Z0, speed=sp)
        frames[sid] = scenes.render_sequence(sc, K, device=dev).cpu().pin_memory()

    def fn(s, q):
        return frames[s][q % K]

    arr = scenes.poisson_arrivals(len(specs), 30.0, args.serve_seconds, seed=args.seed + 7)
    out = {"workload": "64 camera streams: 16 each 320x240, 640x480, 1280x720, 1920x1080; uint8; "
                       "Poisson arrivals, 30 fps per stream; 4 levels; FOE",
           "offered_pairs_per_s": len(arr) / args.serve_seconds}
    rows = None
    for kind in ("native", "batch", "per_frame"):
        if kind == "batch":
            eng = CudaBatchEngine(1080, 1920, levels, max_batch=len(specs), device=dev)
            srv = Server(eng, 40 << 30, max_batch=len(specs))
        elif kind == "native":
            tuner = CudaBatchEngine(1080, 1920, levels, max_batch=len(specs), device=dev)
            rows = tuner.autotune([(frames[s][0], frames[s][1]) for s, *_ in specs])
            del tuner
            eng = srv = NativeServer(1080, 1920, levels, 40 << 30, max_batch=len(specs), rows_per_tile=rows)
        else:
            eng = PerFrameEngine(1080, 1920, levels, device=dev)
            srv = Server(eng, 40 << 30, max_batch=1)
        if kind == "batch":
            eng.set_plan(rows)
        for sid, H, W, *_ in specs:
            assert srv.admit(sid, H, W)
        saturate(srv, fn, ticks=3 if kind == "batch" else 3 * len(specs))      # warm-up
        base = dict(srv.stats)
        t0 = time.perf_counter()
        done = replay(srv, arr, fn)
        dt = time.perf_counter() - t0
        ticks = srv.stats["ticks"] - base.get("ticks", 0)
        res = latency_summary(done)
        res.update({"served_pairs_per_s": res["n"] / dt, "ticks": ticks,
                    "mean_pairs_per_tick": res["n"] / max(ticks, 1),
                    "dropped_frames": srv.stats["dropped_frames"] - base.get("dropped_frames", 0)})
        nt = 100 * len(specs) // 8 if kind == "per_frame" else 100
        l0 = getattr(eng, "launches", 0)
        t0 = time.perf_counter()
        sat = saturate(srv, fn, ticks=nt)
        dt = time.perf_counter() - t0
        npairs = sum(1 for c in sat if c.records is not None)
        res["saturated_pairs_per_s"] = npairs / dt
        if kind != "native":
            res["saturated_launches_per_pair"] = (eng.launches - l0) / max(npairs, 1)
        if kind != "per_frame":
            res["rows_per_tile_per_level"] = rows
            res["hbm_bytes_admitted"] = srv.used
        out[kind] = res
        if kind == "native":
            # the library's own load generator: every stream always has a frame waiting
            # (no Python per frame), so the rate is the runtime's and the device's
            drv = srv.drive({sid: list(frames[sid]) for sid, *_ in specs}, pairs=200 * len(specs))
            px = sum(H * W for _, H, W, *_ in specs) / len(specs)
            # every pair uploads one new frame: the upload rate against one host-to-device
            # copy of a tick's bytes from page-locked memory (the host link's rate)
            tick_bytes = sum(frames[sid][0].numel() * frames[sid][0].element_size() for sid, *_ in specs)
            link = h2d_link_gbs(dev, tick_bytes)
            up = drv["pairs"] / drv["seconds"] * tick_bytes / len(specs) / 1e9
            res["driven"] = {"pairs_per_s": drv["pairs"] / drv["seconds"], "p50_ms": drv["p50_ms"],
                             "p99_ms": drv["p99_ms"], "pairs": drv["pairs"],
                             "gpx_per_s": drv["pairs"] / drv["seconds"] * px / 1e9,
                             "upload_bytes_per_tick": tick_bytes, "upload_gbs": up, "h2d_copy_gbs": link,
                             "frac_of_h2d_copy": up / link,
                             "driver": "ttc_server_drive (native loop, one waiting frame per stream)"}
            srv.close()
        del srv, eng
        torch.cuda.synchronize(dev)
    out["batch_vs_per_frame_saturated"] = out["batch"]["saturated_pairs_per_s"] / out["per_frame"]["saturated_pairs_per_s"]
    out["native_vs_per_frame_saturated"] = (out["native"]["saturated_pairs_per_s"] /
                                            out["per_frame"]["saturated_pairs_per_s"])
    # admission under a small budget: fixed workspace plus room for about 20 streams
    eng = CudaBatchEngine(1080, 1920, levels, max_batch=len(specs), device=dev)
    per = [eng.stream_bytes(H, W) for _, H, W, *_ in specs]
    budget = eng.fixed_bytes() + int(sum(per[:20]))
    srv = Server(eng, budget, max_batch=len(specs))
    admitted = sum(srv.admit(sid, H, W) for sid, H, W, *_ in specs)
    out["admission_small_budget"] = {"budget_bytes": budget, "admitted": int(admitted),
                                     "rejected": int(srv.stats["rejected_streams"]), "bytes_admitted": srv.used}
    return out


def accuracy(sc, res, levels):
    import paper_1612_08825_gb300 as ft
    import scenes
    npairs = res.shape[0]
    gt = np.array([scenes.ground_truth(sc, t + 0.5) for t in range(npairs)])
    out = {"ttc_mse_per_level": [], "foe_mse_px2_per_level": []}
    for l in range(levels):
        r = res[:, l]
        out["ttc_mse_per_level"].append(float(np.mean((r["ttc"] - gt[:, 0]) ** 2)))
        out["foe_mse_px2_per_level"].append(float(np.mean((r["x0"] - gt[:, 1]) ** 2 + (r["y0"] - gt[:, 2]) ** 2)))
    for rule in (0, 1):
        chosen = np.array([ft.select_level(res[t], rule) for t in range(npairs)])
        ttc = np.array([res[t, c]["ttc"] if c >= 0 else np.nan for t, c in enumerate(chosen)])
        foe = np.array([(res[t, c]["x0"], res[t, c]["y0"]) if c >= 0 else (np.nan, np.nan)
                        for t, c in enumerate(chosen)])
        out[f"ttc_mse_rule{rule}"] = float(np.nanmean((ttc - gt[:, 0]) ** 2))
        out[f"foe_mse_px2_rule{rule}"] = float(np.nanmean((foe[:, 0] - gt[:, 1]) ** 2 + (foe[:, 1] - gt[:, 2]) ** 2))
        out[f"levels_chosen_rule{rule}"] = np.bincount(chosen[chosen >= 0], minlength=levels).tolist()
    out["ttc_gt_range"] = [float(gt[:, 0].min()), float(gt[:, 0].max())]
    return out


# FP32 lane-operations the method needs per level-0 cube in this formulation (Sec. II,
# V-A): exact float of the two new pixels (2), per-column sums/differences (2 + 3),
# Ex/Ey/Et (3), G (2), the ten products (10), plus the next pyramid level (2x2 block
# sums of both frames: 6 adds per 4 level-0 pixels = 1.5)
OPS_PER_CUBE0 = 23.5
# DRAM bytes (read + write) of one level-0 launch over the 299 pairs, from an ncu capture
# of the same kernel on an 80-frame video (287.9 MB for 79 pairs: 3.64 MB per pair,
# scaled by pairs)
L0_TRAFFIC_PER_PAIR = 3.64e6


def alu_roof(dev):
    """FP32 issue roof in lane-ops/s: SMs x 128 FP32 lanes x the maximum SM clock."""
    import torch
    _, sm_max, _ = _peaks()
    return torch.cuda.get_device_properties(dev).multi_processor_count * 128 * sm_max * 1e6


def conv_hbm_summary(rows, hbm_peak):
    """The memory-bound FastConv rows on batches of 16 1080p FP32 images (direct path with
    kernels of at most 5 x 5, separable path) as GB/s and fractions of the measured HBM
    copy rate."""
    out = []
    for r in rows:
        if r.get("input") != [16, 1080, 1920] or "input_dtype" in r:
            continue
        ks = r.get("kernel", [0, 9, 9])
        sep = r.get("path") == "separable"
        if sep or ("path" not in r and ks[-1] <= 5):
            out.append({"workload": "16 x 1080 x 1920 FP32 * 1 x %d x %d%s" % (ks[1], ks[2], " (separable)" if sep else ""),
                        "GBps": r["GBps"], "frac": r["hbm_frac"], "us": r["us"]})
    return {"peak": hbm_peak, "unit": "GB/s", "peak_source": "measured HBM copy rate", "rows": out}


def host_cpu():
    """Host core count and CPU model name (for the CPU baseline's record)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        for key in ("model name", "Model name", "cpu model"):
            for line in txt.splitlines():
                if line.split(":")[0].strip() == key:
                    model = line.split(":", 1)[1].strip()
                    break
            if model:
                break
        if not model:
            impl = [l.split(":", 1)[1].strip() for l in txt.splitlines() if l.startswith("CPU implementer")]
            part = [l.split(":", 1)[1].strip() for l in txt.splitlines() if l.startswith("CPU part")]
            if impl and part:
                model = f"Arm CPU implementer {impl[0]} part {part[0]}"
    except OSError:
        pass
    return {"nproc": os.cpu_count() or 1, "model": model or "unknown"}


def rank_env():
    """(world, rank, local rank) from the torch.distributed launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def unit_seed(base: int, rank: int) -> int:
    """Seed of a rank's own video: ranks process independent units (weak scaling)."""
    return base + rank


def whole_job_rate(elapsed_s: float, units_per_rank: int, device) -> tuple:
    """Max-over-ranks elapsed time and the whole-job throughput (units of all ranks / that
    time); the only cross-rank operation besides the barriers."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    world = 1
    if dist.is_available() and dist.is_initialized():
        world = dist.get_world_size()
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return tmax, units_per_rank * world / tmax


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1612_08825_gb300 as ft
    import scenes

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ft.load()
    hbm_peak, sm_max, peak_src = _peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    alu_peak = n_sm * 128 * sm_max * 1e6          # FP32 lane-ops/s at the maximum SM clock

    frames_n = args.frames
    npairs = frames_n - 1
    # every rank works on its own video (independent pairs: weak scaling)
    sc = scenes.tilted_plane_scene(H=H, W=W, seed=unit_seed(args.seed, rank))
    frames = scenes.render_sequence(sc, frames_n, device=dev)
    ctx = ft.TtcContext(H, W, LEVELS, npairs, device=dev)
    out = ctx.new_results(npairs * LEVELS)
    s = torch.cuda.current_stream(dev)

    def step():
        ctx.solve_sequence(frames, levels=LEVELS, mode=ft.MODE_FOE, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    launches_per_step = ctx.last_launch_count

    # level-0 pass timing: events recorded by the library around its launches
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for a, b in ev:
        a.record(s)
        b.record(s)
    clocks = ClockSampler(_smi_index(local))
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(s)
    for i in range(args.steps):
        ctx.set_level0_events(ev[i][0], ev[i][1])
        step()
    end.record(s)
    torch.cuda.synchronize(dev)
    ctx.set_level0_events(None, None)
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    elapsed = start.elapsed_time(end) * 1e-3
    l0_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    tmax, value = whole_job_rate(elapsed, npairs * args.steps, dev)

    res = ft.results_to_numpy(out).reshape(npairs, LEVELS)

    # parity spot check of the timed results and the CPU baseline (rank 0): the oracle
    # on the first pairs of the same video, one host core, bounded time
    parity = None
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        host = frames[: min(frames_n, args.cpu_pairs + 1)].cpu().numpy()
        worst = 0.0
        t0 = time.perf_counter()
        n_done = 0
        for t in range(min(args.cpu_pairs, host.shape[0] - 1)):
            ref = oracle.ttc_pair(host[t], host[t + 1], levels=LEVELS, mode=1)
            n_done += 1
            for l in range(LEVELS):
                err = np.abs(res[t, l]["sums"] - ref[l]["sums"]) / np.maximum(ref[l]["abssums"], 1e-300)
                worst = max(worst, float(err.max()))
            if time.perf_counter() - t0 > args.cpu_seconds:
                break
        dt_cpu = time.perf_counter() - t0
        info = host_cpu()
        cpu = {"value": n_done / dt_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n_done} pairs of the same video, 5 levels, FOE, single thread",
               "us_per_pair": dt_cpu / max(n_done, 1) * 1e6, "nproc": info["nproc"], "cpu_model": info["model"]}
        # the same oracle, one pair per process at a time, over all host cores
        nw = info["nproc"]
        npar = min(host.shape[0] - 1, 2 * nw)
        _, dt_par = oracle.ttc_pairs_parallel(host, npar, LEVELS, 1, nw)
        cpu["all_cores"] = {"value": npar / dt_par, "unit": UNIT, "cores": nw, "kind": "oracle",
                            "sample": f"first {npar} pairs of the same video over {nw} spawned processes"}
        parity = {"pairs_checked": n_done, "max_sum_err_rel_abssum": worst, "tolerance": SUM_TOL_U8}

    # e2e through the public API with pinned host frames: H2D of the video (in chunks
    # that overlap the compute), both stages, D2H of the result records, every step
    e2e = None
    if not args.no_e2e:
        host_frames = frames.cpu().pin_memory()
        hout = torch.empty(npairs * LEVELS * ft.RESULT_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        for _ in range(2):
            ctx.solve_sequence(host_frames, levels=LEVELS, mode=ft.MODE_FOE, out=hout)
        torch.cuda.synchronize(dev)
        k2 = max(3, args.steps // 4)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0.record(s)
        for _ in range(k2):
            ctx.solve_sequence(host_frames, levels=LEVELS, mode=ft.MODE_FOE, out=hout)
        e1.record(s)
        torch.cuda.synchronize(dev)
        _, e2e_rate = whole_job_rate(e0.elapsed_time(e1) * 1e-3, npairs * k2, dev)
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": ft.TtcContext.host_upload_bytes(frames_n, H * W, npairs),
               "d2h_bytes_per_step": int(hout.numel()),
               "steps": k2}
        e2e_res = ft.results_to_numpy(hout).reshape(npairs, LEVELS)
        assert e2e_res.tobytes() == res.tobytes(), "host-buffer path disagrees with device path"

    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_bench(dev, args)

    small = small_bench(dev) if rank == 0 else None

    serve = None
    if rank == 0 and not args.no_serve:
        serve = serve_bench(dev, args)

    conv_rows = None
    grad_rows = None
    if rank == 0 and not args.no_conv:
        conv_rows, _ = fastconv_sweep(dev, hbm_peak, 2.0 * alu_peak, reps=args.conv_reps)
        grad_rows = gradient_bench(dev, hbm_peak, reps=args.conv_reps)

    if rank == 0:
        cubes0 = (H - 1) * (W - 1) * npairs
        achieved_ops = cubes0 * OPS_PER_CUBE0 / (l0_ms * 1e-3)
        # level-0 pass bytes: every frame read once, the level-1 images written
        # (uint16), the tile partials written
        l0_bytes = frames_n * H * W + frames_n * (H // 2) * (W // 2) * 2 + npairs * (-(-(H - 1) // 64)) * (-(-(W - 1) // 256)) * 10 * 4
        step_bytes = frames_n * H * W + npairs * LEVELS * ft.RESULT_DTYPE.itemsize
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": _config(frames_n),
            "roofline": {"kernel": "ttc level-0 pass (ttc_pass_tma_kernel: persistent, TMA-fed, uint8 frames)",
                         "bound": "alu", "achieved": achieved_ops / 1e12, "peak": alu_peak / 1e12,
                         "unit": "TFP32-lane-op/s", "frac": achieved_ops / alu_peak,
                         "traffic": L0_TRAFFIC_PER_PAIR * npairs,
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, 80-frame "
                                           "capture scaled to the launch's pairs",
                         "ops_per_cube": OPS_PER_CUBE0, "cubes_per_launch": cubes0, "launch_ms": l0_ms,
                         "peak_source": f"{n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz ({peak_src} max clock)",
                         "hbm": {"achieved": l0_bytes / (l0_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": l0_bytes / (l0_ms * 1e-3) / 1e9 / hbm_peak, "bytes": l0_bytes}},
            "step_hbm": {"algorithmic_bytes": step_bytes, "GBps": step_bytes / (tmax / args.steps) / 1e9,
                         "frac": step_bytes / (tmax / args.steps) / 1e9 / hbm_peak},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "launches_per_step": launches_per_step,
            "clocks": ck,
            "parity": parity,
            "accuracy": accuracy(sc, res, LEVELS),
            "fastconv": conv_rows,
            "gradient": grad_rows,
            "batch_uneven": batch,
            "serve": serve,
            "plain_ttc_128": small,
        }
        if conv_rows:
            line["fastconv_hbm"] = conv_hbm_summary(conv_rows, hbm_peak)
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=T_FRAMES)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-pairs", type=int, default=120)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-pairs", type=int, default=8)
    ap.add_argument("--conv-reps", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-conv", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=512)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-batch-oracle", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
