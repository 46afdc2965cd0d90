"""Benchmark: ILS smoothing of 1920 x 1080 RGB FP32 frames, N = 4 (the paper's headline size).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one frame through the whole hot path (2N+1 kernels: N fused row
passes, N column passes, one inverse row pass), input already resident in HBM.
The L2 is flushed (a 512 MiB write, then a read of the same buffer) between timed
steps, outside the timed interval.  The headline value times K steps with one event pair per step; the
per-kernel launch times behind the roofline object come from a second loop of
K steps with an event before every launch (those events serialize the launch
queue, so they are kept out of the headline loop).  Prints one JSON line.

--impl reference times the FP64 CPU oracle (the method written out from the
paper, not tuned) on the host cores for the same metric.

Under torchrun (N > 1) every rank smooths its own frames on its own GPU (frames
are independent: replicas, no collective on the data path); the step time is
the max over ranks and the value counts the frames of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ILS 1080p RGB fps & % HBM roofline; learned warm-start vs plain at equal error"
H, W, C = 1080, 1920, 3
LAM, P, EPS, N_ITERS = 1.0, 0.8, 1e-4, 4
SEED = 2000


def bytes_model(H, W, C, N):
    """Algorithmic HBM bytes of the fused design per launch kind and per frame.

    Per channel: P = 4HW bytes (image), S = 4HW bytes (packed half spectrum).
    first row pass reads f, writes S; later row passes read S and f, write S;
    each column pass reads and writes S; the inverse row pass reads S, writes u.
    """
    px = H * W * C
    per = {"row_first": 8 * px, "row": 12 * px, "column": 8 * px, "row_inverse": 8 * px}
    total = (N + 1) * 4 * px + 4 * N * 4 * px
    return per, total


class L2Flush:
    """Evicts the L2 between timed steps: a 512 MiB write (four times the 129 MB L2), then a read
    of the same buffer.  The write alone would leave the L2 full of dirty lines whose write-back
    the next timed step pays for; after the read it holds clean lines of this buffer only, none
    of the step's data."""

    def __init__(self, torch, dev):
        self.buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.buf.zero_()
        self.buf.sum()


def load_capture(kernel: str):
    """The committed ncu counters of `kernel` (profiles/row_pass_traffic.json), or None when there
    are none or the kernel's sources changed since they were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "row_pass_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("kernel") != kernel:
            return None
        for src, digest in d["source_sha256"].items():
            with open(os.path.join(ROOT, src), "rb") as fh:
                if hashlib.sha256(fh.read()).hexdigest() != digest:
                    return None
        return d
    except (OSError, ValueError, KeyError):
        return None


def load_traffic(kernel: str):
    """DRAM bytes (GB) per launch of `kernel` from the committed ncu capture, or None."""
    d = load_capture(kernel)
    return None if d is None else d["traffic_bytes_per_launch"] / 1e9


SMSP_PER_GPU = 152 * 4   # SM sub-partitions: one warp-instruction issue per cycle each


def issue_roof(kernel: str, launch_ms: float, sm_mhz):
    """The launch's warp-instructions (committed ncu count) against the GPU's issue rate at the
    sampled SM clock: the fraction of issue slots the kernel used, the roof its latency-bound
    instruction stream sits under."""
    d = load_capture(kernel)
    if d is None or "warp_instructions_per_launch" not in d or not sm_mhz or launch_ms <= 0:
        return None
    n = float(d["warp_instructions_per_launch"])
    peak = SMSP_PER_GPU * float(sm_mhz) * 1e6   # warp-instructions per second
    return {"warp_instructions_per_launch": n, "peak_warp_instr_per_s": peak,
            "min_launch_us": n / peak * 1e6, "frac": n / (launch_ms / 1000.0) / peak}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def headline_line(ws, steps, warmup, ch, hh, ww, fps, total_ms, pct, prof, e2e_fps, frame_nbytes, clocks) -> dict:
    """The JSON line of the headline measurement: fps of `steps` timed steps over `ws` replicas,
    the dominant kernel's HBM roofline (per-launch event times in `prof`: kind -> (ms, launches))
    and its issue roof, the end-to-end fps, the sampled clocks."""
    per_kind, frame_bytes = bytes_model(hh, ww, ch, N_ITERS)
    peak, peak_kind = load_peaks()
    # dominant kernel = the kind with the largest share of device time
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    achieved = per_kind[dom] / (dom_ms / dom_n / 1000.0) / 1e9
    whole = frame_bytes / (total_ms / steps / 1000.0) / 1e9
    workload = f"ILS {ww}x{hh} {'RGB' if ch == 3 else f'{ch}-channel'} FP32, N=4, lambda=1, p=0.8, eps=1e-4"
    return {
        "metric": METRIC, "value": fps, "unit": "fps", "n_gpus": ws, "steps": steps,
        "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload,
                   "global_batch": ws, "parallelism": f"replicas x{ws}",
                   "l2": "flushed (512 MiB write + read) between timed steps",
                   "mpix_per_s": fps * hh * ww / 1e6},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": load_traffic(dom),
                     "issue": issue_roof(dom, dom_ms / dom_n, clocks.get("sm_mhz")),
                     "traffic_unit": "GB per launch (ncu dram read + write)",
                     "launch_timing": "events around every launch, second loop of the same K steps",
                     "algorithmic_bytes_per_launch": per_kind[dom],
                     "whole_step_gbs": whole, "whole_step_frac": whole / peak,
                     "model": "fused: (20N+4) B per pixel and channel; an unfused stencil / FFT / "
                              "solve / IFFT sequence would move ~28 B per pixel, channel and iteration"},
        "step_ms_p10_p50_p90": [float(v) for v in pct],
        "kernels": {k: {"launches": v[1], "ms_total": v[0], "share": v[0] / max(1e-9, sum(x[0] for x in prof.values()))}
                    for k, v in prof.items()},
        "e2e": None if e2e_fps is None else {"value": e2e_fps, "unit": "fps",
                                              "h2d_bytes_per_step": frame_nbytes,
                                              "d2h_bytes_per_step": frame_nbytes},
        "gpu_launches": sum(v[1] for v in prof.values()),
        "clocks": clocks,
    }


def max_over_ranks(value: float, ws: int, device) -> float:
    """The largest `value` over the ranks (the slowest replica sets a weak-scaling run's time);
    `device` is the tensor device of the process group's backend (cuda for nccl, cpu for gloo)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_fps(total_ms_max: float, steps: int, ws: int, channels: int) -> float:
    """Whole-job frames per second of `ws` replicas that each ran `steps` steps of a
    `channels`-channel image (frames counted in C-channel frames), timed by the slowest rank."""
    frames = steps * ws * (channels / C)
    return frames / (total_ms_max / 1000.0)


def make_frame(c=None, h=None, w=None):
    from paper_2003_07504_gb300 import synth
    return synth.preset_image(h or H, w or W, c or C, "hd", SEED)


# ----------------------------------------------------------------------------- reference arm (CPU oracle)

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle as O
    f = make_frame().astype(np.float64)
    # One step = one channel of the frame through the oracle (1/3 of a frame).
    times = []
    for i in range(args.warmup + args.steps):
        ch = i % C
        t0 = time.perf_counter()
        O.ils_channel(f[ch], LAM, P, EPS, N_ITERS)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    fps = (len(times) / C) / total
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "fps", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ILS 1920x1080 RGB FP32, N=4, lambda=1, p=0.8, eps=1e-4", "global_batch": 1,
                   "parallelism": "replicas", "step": "one channel of one frame (1/3 frame)"},
        "cpu_baseline": {"value": fps, "unit": "fps", "cores": cores, "kind": "oracle",
                         "sample": f"{len(times)} channels of a 1920x1080 RGB frame, N=4, FP64 naive-DFT oracle"},
        "e2e": {"value": fps, "unit": "fps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def adjoint_leg(ils, torch, dev, steps):
    """Backward of N=4 ILS w.r.t. f for 16 gray 512 x 512 images (one 16-channel plan):
    forward with checkpoints, then the hand-written adjoint; CUDA events on the stream."""
    from paper_2003_07504_gb300 import synth
    Ca, Ha, Wa = 16, 512, 512
    f = torch.from_numpy(synth.preset_image(Ha, Wa, Ca, "small", 512)).to(dev)
    gu = torch.from_numpy(synth.random_field((Ca, Ha, Wa), seed=513)).to(dev)
    stream = torch.cuda.current_stream()
    with ils.Plan(Ha, Wa, Ca, LAM, P, EPS, N_ITERS) as plan:
        for _ in range(3):
            u, ck = plan.smooth_checkpointed(f)
            plan.backward_ckpt(ck, gu)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd = bwd = 0.0
        for _ in range(steps):
            ev[0].record(stream)
            u, ck = plan.smooth_checkpointed(f)
            ev[1].record(stream)
            plan.backward_ckpt(ck, gu)
            ev[2].record(stream)
            torch.cuda.synchronize()
            fwd += ev[0].elapsed_time(ev[1])
            bwd += ev[1].elapsed_time(ev[2])
    return {"workload": "16 x 512x512 gray FP32, N=4: forward with checkpoints + ils_backward",
            "forward_ckpt_ms": fwd / steps, "backward_ms": bwd / steps,
            "images_per_s_fwd_bwd": Ca / ((fwd + bwd) / steps / 1000.0)}


def _timed_smooth(plan, f, u, torch, steps, flush, warmup=3):
    """Mean ms per plan.smooth over `steps` calls, L2 flushed before each (CUDA events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.smooth(f, out=u)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.smooth(f, out=u)
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def gray_leg(ils, torch, dev, steps, flush):
    """The headline size as one gray channel: 1 x 1080 x 1920, N = 4."""
    f = torch.from_numpy(make_frame(1, H, W)).to(dev)
    u = torch.empty_like(f)
    with ils.Plan(H, W, 1, LAM, P, EPS, N_ITERS) as plan:
        ms = _timed_smooth(plan, f, u, torch, steps, flush)
    _, frame_bytes = bytes_model(H, W, 1, N_ITERS)
    peak, _ = load_peaks()
    return {"workload": "ILS 1920x1080 gray FP32, N=4, lambda=1, p=0.8, eps=1e-4", "fps": 1000.0 / ms, "ms": ms,
            "mpix_per_s": H * W / ms / 1e3, "frac_of_hbm_peak": frame_bytes / (ms / 1000.0) / 1e9 / peak}


def sweep_4k_leg(ils, torch, dev, steps, flush):
    """3840 x 2160 RGB: N in {1, 2, 4, 10} x lambda in {0.5, 1, 2} x p in {0.8, 1.0}."""
    from paper_2003_07504_gb300 import synth
    Hs, Ws = 2160, 3840
    f = torch.from_numpy(synth.preset_image(Hs, Ws, 3, "uhd", 3000)).to(dev)
    u = torch.empty_like(f)
    peak, _ = load_peaks()
    points = []
    for n in (1, 2, 4, 10):
        _, frame_bytes = bytes_model(Hs, Ws, 3, n)
        for lam in (0.5, 1.0, 2.0):
            for p in (0.8, 1.0):
                with ils.Plan(Hs, Ws, 3, lam, p, EPS, n) as plan:
                    ms = _timed_smooth(plan, f, u, torch, steps, flush, warmup=2)
                points.append({"N": n, "lambda": lam, "p": p, "ms": ms, "fps": 1000.0 / ms,
                               "frac_of_hbm_peak": frame_bytes / (ms / 1000.0) / 1e9 / peak})
    return {"workload": "ILS 3840x2160 RGB FP32 sweep, eps=1e-4", "points": points}


def welsch_leg(ils, torch, dev, steps, flush):
    """ILS with the Welsch penalty (Sec. 5) at 1920 x 1080 RGB with the paper's clip-art
    artifact-removal setting (lambda = 20, gamma = 10/255, N = 10) and its texture-smoothing
    iteration count (lambda = 30, N = 15)."""
    f = torch.from_numpy(make_frame(C, H, W)).to(dev)
    u = torch.empty_like(f)
    peak, _ = load_peaks()
    out = {}
    for name, lam, gamma, n in (("clip_art", 20.0, 10 / 255, 10), ("texture", 30.0, 10 / 255, 15)):
        with ils.Plan(H, W, C, lam, N=n, penalty="welsch", gamma=gamma) as plan:
            ms = _timed_smooth(plan, f, u, torch, steps, flush)
        _, frame_bytes = bytes_model(H, W, C, n)
        out[name] = {"lambda": lam, "gamma": gamma, "N": n, "ms": ms, "fps": 1000.0 / ms,
                     "frac_of_hbm_peak": frame_bytes / (ms / 1000.0) / 1e9 / peak}
    # texture smoothing as the paper runs it: Gaussian pre-smoothing (sigma = 1 px) + Welsch ILS
    with ils.Plan(H, W, C, 30.0, N=15, penalty="welsch", gamma=10 / 255) as plan:
        ms = _timed(lambda: plan.smooth_presmoothed(f, 1.0, out=u), torch, steps, flush)
    out["texture_presmoothed"] = {"lambda": 30.0, "gamma": 10 / 255, "N": 15, "sigma": 1.0, "ms": ms,
                                  "fps": 1000.0 / ms}
    out["workload"] = "Welsch-penalty ILS, 1920x1080 RGB FP32"
    return out


def hqs_leg(ils, torch, dev, steps, flush):
    """The comparison method of Sec. 3.5, half-quadratic splitting with phi = |x|, at 1920 x 1080
    RGB in the paper's Fig. 11 setting (lambda = 0.25, beta0 = 2 lambda, N = 4; kappa = 2)."""
    f = torch.from_numpy(make_frame(C, H, W)).to(dev)
    u = torch.empty_like(f)
    with ils.Plan(H, W, C, 0.25, N=4, penalty="hqs", kappa=2.0) as plan:
        ms = _timed_smooth(plan, f, u, torch, steps, flush)
    return {"workload": "half-quadratic splitting, phi=|x|, 1920x1080 RGB FP32, lambda=0.25, N=4",
            "ms": ms, "fps": 1000.0 / ms}


def _timed(fn, torch, steps, flush, warmup=3):
    """Mean ms per fn() over `steps` calls, L2 flushed before each (CUDA events)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / steps


def colour_leg(ils, torch, dev, steps, flush):
    """1920 x 1080 RGB, N = 4: luminance-only smoothing (Sec. 3.4 option I: one channel),
    per-channel detail enhancement with k = 3 (the paper's figures), and single-scale HDR tone
    mapping of a 12-stop linear-radiance frame (Sec. 4.2: ILS with p = 1, lambda = 10 on the
    log-luminance, base compressed to s = 0.35), each in one call."""
    f = torch.from_numpy(make_frame(C, H, W)).to(dev)
    out = torch.empty_like(f)
    hdr = torch.exp2(12.0 * (f - 0.5)).contiguous()
    with ils.Plan(H, W, 1, LAM, P, EPS, N_ITERS) as p1:
        ms_l = _timed(lambda: p1.smooth_luma(f, 0.0, out=out), torch, steps, flush)
    with ils.Plan(H, W, C, LAM, P, EPS, N_ITERS) as p3:
        ms_e = _timed(lambda: p3.enhance(f, 3.0, out=out), torch, steps, flush)
    with ils.Plan(H, W, 1, 10.0, 1.0, EPS, N_ITERS) as pt:
        ms_t = _timed(lambda: pt.tonemap(hdr, 0.35, 1.0, out=out), torch, steps, flush)
    return {"workload": "1920x1080 RGB FP32, N=4, lambda=1, p=0.8 (tone mapping: lambda=10, p=1)",
            "luma_only": {"ms": ms_l, "fps": 1000.0 / ms_l},
            "detail_enhance_k3": {"ms": ms_e, "fps": 1000.0 / ms_e},
            "hdr_tonemap_single_scale": {"ms": ms_t, "fps": 1000.0 / ms_t}}


def interleaved_leg(ils, torch, dev, steps, flush):
    """The headline frame stored pixel-interleaved (1080 x 1920 x 3), through ils_smooth_hwc."""
    f = torch.from_numpy(make_frame(C, H, W)).to(dev).permute(1, 2, 0).contiguous()
    u = torch.empty_like(f)
    with ils.Plan(H, W, C, LAM, P, EPS, N_ITERS) as plan:
        ms = _timed(lambda: plan.smooth_hwc(f, out=u), torch, steps, flush)
    return {"workload": "ILS 1080x1920x3 (interleaved) FP32, N=4, lambda=1, p=0.8", "ms": ms, "fps": 1000.0 / ms}


BATCH_SIZES = ((480, 640), (720, 1280), (1080, 1920), (1536, 2048))


def batch_leg(ils, torch, dev, steps, flush):
    """64 RGB frames, sizes drawn uniformly from BATCH_SIZES, per-frame lambda ~ U(0.5, 2),
    p in {0.8, 1.0}, N = 4, autotuned kernels, one CUDA-graph launch per step."""
    from paper_2003_07504_gb300 import synth
    rng = np.random.default_rng(4000)
    frames, px = [], 0
    for k in range(64):
        hh, ww = BATCH_SIZES[rng.integers(len(BATCH_SIZES))]
        lam = float(rng.uniform(0.5, 2.0))
        p = float(rng.choice([0.8, 1.0]))
        f = torch.from_numpy(synth.preset_image(hh, ww, 3, "hd", 4000 + k)).to(dev)
        frames.append((f, torch.empty_like(f), lam, p, EPS, N_ITERS))
        px += hh * ww
    stream = torch.cuda.current_stream()
    with ils.Batch(frames, autotune=True) as b:
        for _ in range(3):
            b.run()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            b.run()
            s1.record(stream)
            torch.cuda.synchronize()
            tot += s0.elapsed_time(s1)
    ms = tot / steps
    # the same frames as one plan call each, one after another on one stream (plans made and
    # warmed up beforehand, graph replay per plan): what the batch's concurrent branches gain
    plans = [ils.Plan(f.shape[1], f.shape[2], 3, lam, p, eps, n) for f, _, lam, p, eps, n in frames]
    for pl, (f, u, *_) in zip(plans, frames):
        for _ in range(3):
            pl.smooth(f, out=u)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for pl, (f, u, *_) in zip(plans, frames):
            pl.smooth(f, out=u)
        s1.record(stream)
        torch.cuda.synchronize()
        tot += s0.elapsed_time(s1)
    for pl in plans:
        pl.close()
    serial_ms = tot / steps
    # what a persistent work-queue kernel could reach at best: every frame at its size class's
    # saturated rate, measured as one 24-channel plan call per class (the passes fill the GPU,
    # so fill, drain and launch gaps are small against the work), summed over the batch
    per_px = {}
    for hh, ww in BATCH_SIZES:
        fc = torch.from_numpy(synth.preset_image(hh, ww, 24, "hd", 4100)).to(dev)
        uc = torch.empty_like(fc)
        with ils.Plan(hh, ww, 24, 1.0, 0.8, EPS, N_ITERS) as pl:
            per_px[(hh, ww)] = _timed_smooth(pl, fc, uc, torch, max(3, steps), flush) / (24 * hh * ww)
        del fc, uc
    bound_ms = sum(per_px[(f.shape[1], f.shape[2])] * 3 * f.shape[1] * f.shape[2] for f, *_ in frames)
    nbytes = sum(bytes_model(f.shape[1], f.shape[2], 3, N_ITERS)[1] for f, *_ in frames)
    peak, _ = load_peaks()
    return {"workload": "64 RGB FP32 frames, sizes uniform over 640x480 / 1280x720 / 1920x1080 / 2048x1536, "
                        "lambda~U(0.5,2), p in {0.8,1}, N=4, one graph launch",
            "ms_per_batch": ms, "frames_per_s": 64 / (ms / 1000.0), "mpix_per_s": px / (ms / 1000.0) / 1e6,
            "algorithmic_gbs": nbytes / (ms / 1000.0) / 1e9, "frac_of_hbm_peak": nbytes / (ms / 1000.0) / 1e9 / peak,
            "frames_one_after_another_ms": serial_ms,
            "saturated_class_bound_ms": bound_ms,
            "saturated_us_per_mpix_channel": {f"{hh}x{ww}": 1e9 * v for (hh, ww), v in per_px.items()},
            "note": "frames_one_after_another_ms: the same 64 frames as 64 plan calls on one stream; "
                    "saturated_class_bound_ms: sum over the frames of 3 H W x the per-pixel time of a "
                    "24-channel plan call of the frame's size (a persistent kernel's best case)"}


def batch_4k_leg(ils, torch, dev, steps, flush):
    """8 RGB 3840 x 2160 frames with the larger iteration counts (N = 10 and 15, alternating),
    lambda ~ U(0.5, 2), p in {0.8, 1.0}, autotuned kernels, one CUDA-graph launch per step."""
    from paper_2003_07504_gb300 import synth
    rng = np.random.default_rng(4100)
    Hs, Ws = 2160, 3840
    base = torch.from_numpy(synth.preset_image(Hs, Ws, 3, "uhd", 4100)).to(dev)
    frames, nbytes = [], 0
    for k in range(8):
        n = 10 if k % 2 == 0 else 15
        f = torch.roll(base, shifts=(97 * k, 211 * k), dims=(1, 2)).contiguous()
        frames.append((f, torch.empty_like(f), float(rng.uniform(0.5, 2.0)), float(rng.choice([0.8, 1.0])), EPS, n))
        nbytes += bytes_model(Hs, Ws, 3, n)[1]
    with ils.Batch(frames, autotune=True) as b:
        ms = _timed(b.run, torch, steps, flush, warmup=2)
    peak, _ = load_peaks()
    return {"workload": "8 RGB FP32 frames 3840x2160, N in {10, 15}, lambda~U(0.5,2), p in {0.8,1}, one graph launch",
            "ms_per_batch": ms, "frames_per_s": 8 / (ms / 1000.0), "mpix_per_s": 8 * Hs * Ws / (ms / 1000.0) / 1e6,
            "algorithmic_gbs": nbytes / (ms / 1000.0) / 1e9, "frac_of_hbm_peak": nbytes / (ms / 1000.0) / 1e9 / peak}


CNN_FLOP_PER_PX = 2 * 9 * (3 * 32 + 4 * 32 * 32 + 32 * 3)  # 77,184: six 3x3 convolutions per pixel


def training_leg(torch, dev, steps):
    """One training step of the warm-start network on 16 RGB 256 x 256 crops: targets by plain
    ILS N=4 (this library), forward, MSE, backward (input and weight gradients), Adam.  The
    network FLOPs are 3 x 77,184 per pixel (forward, input gradients, weight gradients)."""
    from paper_2003_07504_gb300 import ils, synth, warmstart as ws
    B, S = 16, 256
    f = torch.from_numpy(synth.preset_image(S, S, 3 * B, "small", 6000).reshape(B, 3, S, S)).to(dev)
    target, grad = torch.empty_like(f), torch.empty_like(f)
    loss = torch.zeros(1, device=dev)
    net = ws.WarmStartNet(B * S * S, ws.init_params(seed=1))
    stream = torch.cuda.current_stream()
    with ils.Plan(S, S, 3 * B, LAM, P, EPS, N_ITERS) as plan:
        def step():
            plan.smooth(f.view(3 * B, S, S), out=target.view(3 * B, S, S))
            loss.zero_()
            u0 = net.forward(f)
            ws.mse(u0, target, grad, loss)
            net.zero_grad()
            net.backward(f, grad)
            net.adam_step(1e-4)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        net.check()
    net.close()
    tflops = 3 * CNN_FLOP_PER_PX * B * S * S / (ms / 1000.0) / 1e12
    return {"workload": "16 x 3 x 256 x 256 crops: ILS N=4 targets + network forward/backward + Adam",
            "ms_per_step": ms, "crops_per_s": B / (ms / 1000.0), "network_tflops_incl_targets": tflops}


def warm_leg(torch, dev, steps, flush):
    """Learned warm start vs plain ILS at 1920x1080 RGB (lambda=1, p=0.8): fps of the whole
    warm path (network + 1 or 2 ILS iterations + the iterate-change check and fallback
    decision) against plain N=4 on one frame, and the RMS distance to converged ILS from f
    (ILS iterated until the largest per-iteration change is < 1e-6, capped at 2000) averaged
    over three fresh frames, with the fallback count."""
    from paper_2003_07504_gb300 import ils, synth, warmstart as ws
    path = ws.DEFAULT_WEIGHTS
    if not os.path.exists(path):
        return {"unavailable": "no trained weights file"}
    seeds = (90004, 90005, 90006)
    frames = [torch.from_numpy(synth.preset_image(H, W, C, "hd", sd)).to(dev) for sd in seeds]
    net = ws.WarmStartNet(H * W, ws.load_params(path))
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / steps

    refs = [ws.converged_ils(lambda h, w, c, n: ils.Plan(h, w, c, LAM, P, EPS, n), f, max_iters=20000) for f in frames]
    rms = lambda u, k: float(((u - refs[k][0]) ** 2).mean().sqrt())
    f = frames[0]
    out = {"workload": "1920x1080 RGB, lambda=1, p=0.8, eps=1e-4; reference = ILS from f iterated until the "
                       "largest per-iteration change is < 1e-6 (about 10,000 iterations at 1080p; cap 20,000); errors averaged over 3 frames, "
                       "timing on the first",
           "reference_iterations": [r[1] for r in refs],
           "reference_last_change": [r[2] for r in refs],
           "reference_stationarity_residual": [ws.stationarity_residual(r[0], fk, LAM, P, EPS)
                                               for r, fk in zip(refs, frames)],
           "residual_of_f": [ws.stationarity_residual(fk, fk, LAM, P, EPS) for fk in frames],
           "uses_tcgen05": net.uses_tcgen05}
    u0 = torch.empty_like(f).view(1, C, H, W)
    net_ms = timed(lambda: net.infer(f.view(1, C, H, W), out=u0))
    tflops = CNN_FLOP_PER_PX * H * W / (net_ms / 1000.0) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
    out["network"] = {"ms": net_ms, "flop_per_px": CNN_FLOP_PER_PX, "tflops": tflops,
                      "frac_of_bf16_peak": tflops / float(peaks["bf16_tflops"]),
                      "kernels": "six tcgen05 convolution launches (layer by layer; ILS_CNN_FUSED=1: two fused kernels)" if net.uses_tcgen05 else "mma.sync"}
    with ils.Plan(H, W, C, LAM, P, EPS, N_ITERS) as p4:
        errs = [rms(p4.smooth(fk), k) for k, fk in enumerate(frames)]
        u4 = torch.empty_like(f)
        ms = timed(lambda: p4.smooth(f, out=u4))
        out["plain_N4"] = {"fps": 1000.0 / ms, "ms": ms, "rms_to_converged": float(np.mean(errs)),
                           "rms_per_frame": errs}
    for iters in (1, 2):
        sm = ws.WarmSmoother(net, H, W, C, LAM, P, EPS, iters=iters, n_plain=N_ITERS, tau=ws.DEFAULT_TAU)
        errs, fbs, deltas = [], 0, []
        for k, fk in enumerate(frames):
            u, fb, d = sm.smooth(fk)
            errs.append(rms(u, k))
            fbs += int(fb)
            deltas.append(d)
        u = torch.empty_like(f)
        res = {"rms_to_converged": float(np.mean(errs)), "rms_per_frame": errs, "fallbacks": fbs,
               "frames": len(frames), "last_change": deltas,
               "timing": "one CUDA graph per call: network, warm iterations with the change reduced in the final "
                         "pass, device-side fallback decision (conditional node); no host wait"}
        res["ms"] = timed(lambda: sm.smooth_async(f, out=u))
        res["fps"] = 1000.0 / res["ms"]
        out[f"warm_{iters}_iter"] = res
        sm.close()
    net.check()
    net.close()
    return out


def cpu_baseline_sample(runs: int = 3):
    """The oracle as it stands (FP64, naive separable DFT, untuned) on the host cores: the median
    of `runs` runs of one channel of the 1080p frame (N=4), scaled to RGB fps (a frame is three
    independent channels) and to gray fps, plus the 256 x 256 gray parity image (N=4)."""
    import statistics

    import oracle as O
    from paper_2003_07504_gb300 import synth
    f = make_frame()[0].astype(np.float64)
    O.ils_channel(f[:64, :64], LAM, P, EPS, 1)   # warm the imports
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        O.ils_channel(f, LAM, P, EPS, N_ITERS)
        ts.append(time.perf_counter() - t0)
    med = statistics.median(ts)
    g = synth.preset_image(256, 256, 1, "small", SEED)[0].astype(np.float64)
    ts1 = []
    for _ in range(runs):
        t0 = time.perf_counter()
        O.ils_channel(g, LAM, P, EPS, N_ITERS)
        ts1.append(time.perf_counter() - t0)
    return {"value": (1.0 / C) / med, "unit": "fps", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"median of {runs} runs of one 1920x1080 channel, N=4, FP64 naive-DFT oracle "
                      f"(RGB fps = 1/3 frame / time)",
            "runs_s": ts, "gray_1080p_fps": 1.0 / med,
            "parity_256x256_gray_ms": 1000.0 * statistics.median(ts1)}


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2003_07504_gb300 import build
    if rank == 0 or ws == 1:
        build.build()
    if ws > 1:
        dist.barrier()
    from paper_2003_07504_gb300 import ils

    ch, hh, ww = args.channels, args.height, args.width
    frame = make_frame(ch, hh, ww)
    f = torch.from_numpy(frame).to(dev)
    u = torch.empty_like(f)
    flush = L2Flush(torch, dev)
    plan = ils.Plan(hh, ww, ch, LAM, P, EPS, N_ITERS)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.smooth(f, out=u)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        # the same calls, untimed, for ~0.5 s before the timed steps: the clock sampler (one
        # sample per 200 ms) sees the GPU under this load, not only across the short timed region
        t_settle = time.perf_counter()
        while time.perf_counter() - t_settle < 0.5:
            for _ in range(20):
                flush()
                plan.smooth(f, out=u)
            torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush()
            starts[i].record(stream)
            plan.smooth(f, out=u)
            ends[i].record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        # per-kernel launch durations (CUDA events on the launching stream around every launch)
        plan.set_profiling(True)
        for i in range(args.steps):
            flush()
            plan.smooth(f, out=u)
        torch.cuda.synchronize()
        prof = plan.profile()
        plan.set_profiling(False)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    pct = np.percentile(step_ms, [10, 50, 90]) if step_ms else [0.0, 0.0, 0.0]
    # headline: the median step (robust to the pool's occasional slow launch), the slowest
    # rank's median for N > 1; the mean-based rate is reported beside it
    mean_total_ms = max_over_ranks(sum(step_ms), ws, dev)
    total_ms = max_over_ranks(float(np.median(step_ms)) * args.steps, ws, dev)
    frames = args.steps * ws * (ch / C)   # frames of C channels
    fps = replica_fps(total_ms, args.steps, ws, ch)
    fps_mean = replica_fps(mean_total_ms, args.steps, ws, ch)

    # end to end through the host-buffer entry point: pinned input, H2D + kernels + D2H per step
    e2e_fps = None
    if not args.no_e2e:
        fh = torch.from_numpy(frame).pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        for _ in range(2):
            plan.smooth_host(fh, uh)
        e2e_times = []
        for _ in range(args.steps):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.smooth_host(fh, uh)
            e2e_times.append(time.perf_counter() - t0)
        e2e_fps = frames / max_over_ranks(sum(e2e_times), ws, dev)

    if rank == 0:
        line = headline_line(ws=ws, steps=args.steps, warmup=args.warmup, ch=ch, hh=hh, ww=ww, fps=fps,
                             total_ms=total_ms, pct=pct, prof=prof, e2e_fps=e2e_fps, frame_nbytes=int(frame.nbytes),
                             clocks=clk.summary())
        line["value_stat"] = "median of the timed steps (steps x median step time for ms_per_step)"
        line["fps_mean"] = fps_mean
        if not args.no_extras:
            ksteps = max(3, min(args.steps, 10))
            line["gray"] = gray_leg(ils, torch, dev, ksteps, flush)
            line["welsch"] = welsch_leg(ils, torch, dev, ksteps, flush)
            line["colour"] = colour_leg(ils, torch, dev, ksteps, flush)
            line["interleaved"] = interleaved_leg(ils, torch, dev, ksteps, flush)
            line["hqs"] = hqs_leg(ils, torch, dev, ksteps, flush)
            line["sweep_4k"] = sweep_4k_leg(ils, torch, dev, 5, flush)
            line["adjoint"] = adjoint_leg(ils, torch, dev, max(3, min(args.steps, 20)))
            line["batch"] = batch_leg(ils, torch, dev, max(3, min(args.steps, 10)), flush)
            line["batch_4k_large_n"] = batch_4k_leg(ils, torch, dev, 3, flush)
            line["warm_start"] = warm_leg(torch, dev, max(3, min(args.steps, 10)), flush)
            line["training"] = training_leg(torch, dev, max(3, min(args.steps, 10)))
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_sample()
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # profiling variants (not the headline workload): other channel counts / sizes, no e2e leg
    ap.add_argument("--channels", type=int, default=C)
    ap.add_argument("--height", type=int, default=H)
    ap.add_argument("--width", type=int, default=W)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint / batch / warm-start legs")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
