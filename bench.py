"""Throughput benchmark of the One-Sided Box Filter library on GB300.

Headline workload: the plain float32 forward on 1 x 3 x 4096 x 4096 synthetic
piecewise-constant + noise images (40 rectangles, 20 triangles, sigma 0.05, each channel
its own plane), r = 8, 30 passes.  A "step" is one full filter call (all 30 passes).
The inputs (201 MB) exceed the 129 MB L2, so no flush is needed between steps.

Printed JSON line (rank 0):
  value        whole-job Mpixel*iter/s (cropped output pixels x passes / time), kernels
               only, inputs already resident in HBM;
  e2e          the same metric through osbf_filter_host() with pinned host buffers
               (host->device copy of the input and device->host copy of the result
               inside the timed region);
  roofline     the forward tile kernel's algorithmic bytes (read + write of every frame
               pixel once per launch) per launch over its average launch time, against
               the measured HBM copy bandwidth;
  cpu_baseline the CPU oracle on the host cores, on a bounded sample (a 1024 x 1024 crop
               of the same image, r = 8) -- a reported baseline, not the target;
  forms        the other forms against the plain one on the same GPU: forward+backward
               (16x3x512^2, r=3, 5 passes), batched (256 images), float16 / bfloat16
               storage (7680x4320x3, r=4, 30 passes; distance of the 16-bit results from
               the float32 results on a sampled region -- the error against the FP64
               oracle at this configuration is measured by the test suite), the fast
               approximation, the 3D filter, the one-sided Gaussian filter, and the
               r x fused-depth sweep at 4096^2 x 3.

`--impl reference` times the CPU oracle as the reference arm (bounded sample per step).
Multi-GPU: `torchrun --nproc-per-node N bench.py --gpus N`: every rank filters its own
batch (weak scaling, no collective on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpixel·iter/s at 4096² r=8 FP32 & % HBM roofline; fwd+bwd and batched vs plain"
UNIT = "Mpixel*iter/s"
N_, C_, H_, W_, R_, ITERS_ = 1, 3, 4096, 4096, 8, 30
WORKLOAD = "osbf forward, 1x3x4096x4096 float32, r=8, 30 passes, piecewise-constant+noise (sigma 0.05)"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes (read + write) of one frame-to-frame launch of the headline workload's tile
# kernel (early loads, 32-byte register stores), from one ncu capture of that launch:
# 204.9 MB read + 161.0 MB written (reset to None whenever that kernel changes)
TRAFFIC_PER_LAUNCH = 366.0e6


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, pg, device=None) -> float:
    """Max of a scalar over all ranks (identity without a process group)."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline_sample(x_plane: np.ndarray, seconds_hint: float = 10.0):
    """The oracle (as it stands) on the host cores: 1024 x 1024 crop, r = 8, enough passes
    for about `seconds_hint` seconds of work.  Returns (Mpixel*iter/s, cores, description,
    near ties): the literal FP32 rule's count of output pixels whose best two |d_i| differ
    by less than 1e-6 in the sample's last pass (taken from the same run's gaps)."""
    import oracle

    crop = np.ascontiguousarray(x_plane[:1024, :1024], dtype=np.float64)
    t0 = time.perf_counter()
    oracle.filter(crop, R_, 1)
    t1 = time.perf_counter() - t0
    iters = max(1, min(ITERS_, int(seconds_hint / max(t1, 1e-3))))
    t0 = time.perf_counter()
    res = oracle.filter(crop, R_, iters, want_gaps=True)
    dt = time.perf_counter() - t0
    mpx = crop.size * iters / dt / 1e6
    ties = int((oracle.crop(res["gaps"][-1], R_) < 1e-6).sum())
    return (mpx, oracle.threads(), f"1 plane, 1024x1024 crop of channel 0, r={R_}, {iters} passes, FP64 direct sums",
            {"count": ties, "pixels": int(crop.size), "pass": iters, "rule": "best two |d_i| within 1e-6 (FP64)"})


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2108_05021_gb300 import synth

    x = synth.piecewise_stack(1, 1, 512, 512, seed=0, sigma=0.05)[0, 0].astype(np.float64)
    iters = 2
    sample = f"per step: 1 plane, 512x512 crop, r={R_}, {iters} passes, FP64 direct sums"
    for _ in range(args.warmup):
        oracle.filter(x, R_, iters)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.filter(x, R_, iters)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = x.size * iters * args.steps / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------------
# the other forms, each against the plain form on the same GPU
# --------------------------------------------------------------------------------------
def _time(fn, steps, warmup=3):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps * 1e-3  # seconds per step


def form_fwd_bwd(dev):
    """16 x 3 x 512^2, r = 3, 5 passes; loss = MSE(osbf(noisy), clean)."""
    import torch

    from paper_2108_05021_gb300 import osbf, synth

    N, C, H, W, r, it = 16, 3, 512, 512, 3, 5
    x = torch.from_numpy(synth.piecewise_stack(N, C, H, W, seed=50, sigma=0.05)).to(dev)
    clean = torch.from_numpy(synth.piecewise_stack(N, C, H, W, seed=50, sigma=0.0)).to(dev)
    maps = torch.empty(osbf.maps_shape(x, r, it), dtype=torch.uint8, device=dev)
    out = torch.empty_like(x)
    gin = torch.empty_like(x)

    def fwd():
        osbf.filter(x, r, it, out=out)

    def fwd_bwd():
        osbf.filter(x, r, it, maps=maps, out=out)
        g = (2.0 / out.numel()) * (out - clean)
        osbf.backward(g, maps, r, it, out=gin)

    def fwd_bwd_ck():
        y, ck = osbf.filter_checkpointed(x, r, it, 2)
        g = (2.0 / y.numel()) * (y - clean)
        osbf.backward_checkpointed(g, ck, r, it, 2)

    units = N * C * H * W * it
    t_f, t_fb, t_ck = _time(fwd, 20), _time(fwd_bwd, 20), _time(fwd_bwd_ck, 10)
    res = {"workload": "16x3x512x512 float32, r=3, 5 passes, MSE(osbf(noisy), clean)",
           "fwd_mpix_iter_s": units / t_f / 1e6, "fwd_bwd_mpix_iter_s": units / t_fb / 1e6,
           "fwd_bwd_checkpointed_k2_mpix_iter_s": units / t_ck / 1e6,
           "fwd_bwd_time_over_fwd": t_fb / t_f}
    # the parts at the 4096 x 4096 x 3 size, 10 passes: plain forward, map-writing forward,
    # backward alone
    xb = torch.from_numpy(synth.piecewise_stack(1, 3, 4096, 4096, seed=51, sigma=0.05)).to(dev)
    ob, gb, gib = torch.empty_like(xb), torch.randn_like(xb), torch.empty_like(xb)
    parts = {}
    for rr in (3, 8):
        mb = torch.empty(osbf.maps_shape(xb, rr, 10), dtype=torch.uint8, device=dev)
        tp = _time(lambda: osbf.filter(xb, rr, 10, out=ob), 5)
        tm = _time(lambda: osbf.filter(xb, rr, 10, maps=mb, out=ob), 5)
        tb = _time(lambda: osbf.backward(gb, mb, rr, 10, out=gib), 5)
        u = xb.numel() * 10 / 1e9
        parts[f"r{rr}"] = {"fwd_gpix_iter_s": u / tp, "fwd_maps_gpix_iter_s": u / tm, "bwd_gpix_iter_s": u / tb}
        del mb
    res["parts_4096x4096x3_10_passes"] = parts
    return res


def form_batched(dev):
    """256 images, H, W ~ U[64, 2048], r in {1,2,3,4,6,8}, passes ~ U[1, 30]."""
    import torch

    from paper_2108_05021_gb300 import osbf, synth

    rng = np.random.default_rng(4)
    ins, rs, its = [], [], []
    for k in range(256):
        H, W = (int(v) for v in rng.integers(64, 2049, size=2))
        ins.append(torch.from_numpy(synth.piecewise_stack(1, 1, H, W, seed=2000 + k, sigma=0.05)[0, 0]).to(dev))
        rs.append(int(rng.choice([1, 2, 3, 4, 6, 8])))
        its.append(int(rng.integers(1, 31)))
    outs = [torch.empty_like(t) for t in ins]
    units = sum(t.numel() * i for t, i in zip(ins, its))

    def batched():
        osbf.batched(ins, rs, its, outputs=outs)

    def plain():
        for t, r, i, o in zip(ins, rs, its, outs):
            osbf.filter(t, r, i, out=o)

    t_b = _time(batched, 5, warmup=2)
    lat = sorted(osbf.batched_latencies(256))
    t_p = _time(plain, 3, warmup=1)
    # the tuned layout policy (job order per pass round, CTAs per SM), timed on this batch
    osbf.autotune_batched(ins, rs, its, outs)
    pol = osbf.batched_policy(ins, rs, its, outs)
    t_t = _time(batched, 5, warmup=2)
    lat_t = sorted(osbf.batched_latencies(256))
    return {"workload": "256 float32 images, H,W~U[64,2048], r in {1,2,3,4,6,8}, passes~U[1,30]",
            "batched_mpix_iter_s": units / t_b / 1e6, "plain_calls_mpix_iter_s": units / t_p / 1e6,
            "batched_over_plain": t_p / t_b, "p50_latency_ms": 1e3 * lat[len(lat) // 2],
            "p99_latency_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "tuned_policy": {"job_order": {1: "by decreasing work", 2: "by radius, then decreasing work"}.get(
                                 pol[0] if pol else 0, "as given"),
                             "ctas_per_sm": pol[1] if pol else None,
                             "batched_mpix_iter_s": units / t_t / 1e6,
                             "p50_latency_ms": 1e3 * lat_t[len(lat_t) // 2],
                             "p99_latency_ms": 1e3 * lat_t[min(len(lat_t) - 1, int(0.99 * len(lat_t)))]},
            "total_pixel_iters": units}


def form_precision(dev):
    """7680 x 4320 x 3 stored as f32 / f16 / bf16, r = 4, 30 passes, sigma 0.03: throughput,
    and the 16-bit results' distance from the float32 results (the error against the FP64
    oracle at this configuration is measured in tests/test_gpu_forward.py)."""
    import torch

    from paper_2108_05021_gb300 import osbf, synth

    H, W, r, it = 4320, 7680, 4, 30
    x32 = synth.piecewise_stack(1, 3, H, W, seed=3, sigma=0.03)
    res = {"workload": "1x3x4320x7680, r=4, 30 passes, sigma 0.03"}
    y0, x0, s = H // 2, W // 2, 48  # sampled output region of plane 0
    ref = None
    maps32 = None
    FW = W + 2 * r
    for name, dt in (("f32", torch.float32), ("f16", torch.float16), ("bf16", torch.bfloat16)):
        xin = x32 if name == "f32" else synth.round_to_storage(x32, name)
        xt = torch.from_numpy(xin).to(dev).to(dt)
        out = torch.empty_like(xt)
        t = _time(lambda: osbf.filter(xt, r, it, out=out), 5)
        got = out[0, 0, y0:y0 + s, x0:x0 + s].float().cpu().numpy()
        res[name] = {"mpix_iter_s": 3 * H * W * it / t / 1e6}
        # selection maps of every pass (not timed): flips against the float32 run
        maps = torch.empty(osbf.maps_shape(xt, r, it), dtype=torch.uint8, device=dev)
        osbf.filter(xt, r, it, maps=maps, out=out)
        if ref is None:
            ref = got
            maps32 = maps
        else:
            d = np.abs(got - ref)
            flips = [int((maps[k, ..., :FW] != maps32[k, ..., :FW]).sum()) for k in range(it)]
            res[name].update({"max_abs_diff_vs_f32": float(d.max()), "mean_abs_diff_vs_f32": float(d.mean()),
                              "diff_sample": f"{s}x{s} at ({y0},{x0}), plane 0",
                              "selection_flips_vs_f32": {"total": sum(flips), "pass_1": flips[0],
                                                         "last_pass": flips[-1],
                                                         "pixel_passes": 3 * (H + 2 * r) * FW * it}})
            del maps
    del maps32
    return res


def form_fast(dev, x):
    """The fast approximation (Algorithm 3, Eq. (app)) on the headline workload (4096^2 x 3,
    r = 8, 30 passes): its throughput next to the exact filter's, and how far its output
    is from the exact filter's (the comparison the paper plots for the fast variant)."""
    import torch

    from paper_2108_05021_gb300 import osbf

    r, it = R_, ITERS_
    o_exact, o_fast = torch.empty_like(x), torch.empty_like(x)
    t_exact = _time(lambda: osbf.filter(x, r, it, out=o_exact), 10)
    t_fast = _time(lambda: osbf.filter_fast(x, r, it, out=o_fast), 10)
    d = (o_fast - o_exact).abs()
    units = x.numel() * it
    return {"workload": f"1x3x4096x4096 float32, r={r}, {it} passes", "fast_mpix_iter_s": units / t_fast / 1e6,
            "exact_mpix_iter_s": units / t_exact / 1e6, "fast_time_over_exact": t_fast / t_exact,
            "mean_abs_diff_vs_exact": float(d.mean()), "max_abs_diff_vs_exact": float(d.max()),
            "pixels_differing_from_exact": float((d > 0).float().mean())}


def form_volume(dev):
    """The 3D filter (Sec. "Higher Dimension Case"): 1 x 1 x 128 x 256 x 256 float32 volume,
    r = 2 (the radius of the paper's volume example), 10 passes."""
    import torch

    from paper_2108_05021_gb300 import osbf, synth

    D, H, W, r, it = 128, 256, 256, 2, 10
    scenes = synth.piecewise_stack(1, 4, H, W, seed=11, sigma=0.0)[0]
    rng = np.random.default_rng(11)
    vol = np.concatenate([np.repeat(scenes[k][None], D // 4, axis=0) for k in range(4)])
    vol = np.clip(vol + rng.normal(0, 0.05, vol.shape), 0, 1).astype(np.float32)[None, None]
    x = torch.from_numpy(vol).to(dev)
    out = torch.empty_like(x)
    t = _time(lambda: osbf.filter3d(x, r, it, out=out), 10)
    units = D * H * W * it
    FD, FH, FW = D + 2 * r, H + 2 * r, W + 2 * r
    return {"workload": f"1x1x{D}x{H}x{W} float32, r={r}, {it} passes", "gvox_iter_s": units / t / 1e9,
            "ms_per_call": t * 1e3,
            # per pass: z-pass reads U, writes Zm, Zp; yx-pass reads U, Zm, Zp and writes U'
            "bytes_per_pass_algorithmic_min": 8 * FD * FH * FW, "bytes_per_pass_two_kernels": 28 * FD * FH * FW}


def form_gauss(dev, x):
    """The one-sided Gaussian filter (Algorithm 1 with the one-sided Gaussian kernels of Sec.
    "Separable Kernels") on the 4096 x 4096 x 3 input: r = 8, sigma = 3 (the paper's sigma
    for its Gaussian comparisons), 10 passes.  Bound by FP32 arithmetic, not HBM: per frame
    pixel and pass the separable sums take 8 (r+1) FMAs (2 (r+1) for Up and Dn, 6 (r+1) for
    the left / right sums of Up, Dn and Fy)."""
    import torch

    from paper_2108_05021_gb300 import osbf

    r, sigma, it = 8, 3.0, 10
    out = torch.empty_like(x)
    t_full = _time(lambda: osbf.filter_gauss(x, r, sigma, it, out=out), 10)
    t_two = _time(lambda: osbf.filter_gauss(x, r, sigma, 2, out=out), 10)
    pass_s = (t_full - t_two) / (it - 2)
    N, C, H, W = x.shape
    frame_px = N * C * (H + 2 * r) * (W + 2 * r)
    flops = 16 * (r + 1) * frame_px
    peak = 152 * 128 * 2 * 2.07e9  # FP32 lanes x 2 flops x maximum SM clock
    return {"workload": f"{N}x{C}x{H}x{W} float32, r={r}, sigma={sigma}, {it} passes",
            "gpix_iter_s": x.numel() * it / t_full / 1e9, "ms_per_call": t_full * 1e3,
            "pass_us": pass_s * 1e6, "pass_flops_algorithmic": flops,
            "achieved_tflops": flops / pass_s / 1e12, "fp32_peak_tflops_max_clock": peak / 1e12,
            "frac_of_fp32_peak": flops / pass_s / peak}


def form_sweep(dev, x):
    """r x fused depth on the tile kernel (the depth actually run, from the launch count: a
    requested depth is clamped to the largest whose tile fits shared memory), the strip kernel,
    and the tuner's choice, at 4096^2 x 3; then a 3 x 256 x 256 image, where launch overheads
    weigh more and fused passes can win."""
    import torch

    from paper_2108_05021_gb300 import osbf, synth

    def sweep(xx, radii, tag):
        out = torch.empty_like(xx)
        N, C, H, W = xx.shape
        rows = []
        for r in radii:
            for D in (1, 2, 4, 8):
                try:
                    t = _time(lambda: osbf.filter(xx, r, ITERS_, depth=D, variant="tile", out=out), 5, warmup=2)
                except osbf.OSBFError:
                    continue
                # depth 1 runs ITERS_ launches (+ a padding launch unless the first pass pads
                # itself); deeper groups always follow a padding launch
                launches = osbf.last_launch_count(dev.index)
                eff = 1 if launches >= ITERS_ else -(-ITERS_ // max(launches - 1, 1))
                rows.append({"input": tag, "r": r, "kernel": "tile", "depth": D, "depth_run": eff,
                             "gpix_iter_s": xx.numel() * ITERS_ / t / 1e9})
            if r <= 8:
                t = _time(lambda: osbf.filter(xx, r, ITERS_, variant="strip", out=out), 5, warmup=2)
                rows.append({"input": tag, "r": r, "kernel": "strip", "depth": 1, "depth_run": 1,
                             "gpix_iter_s": xx.numel() * ITERS_ / t / 1e9})
            osbf.autotune(torch.float32, N * C, H, W, r, ITERS_, device=dev.index)
            d, v = osbf.tuned(torch.float32, N * C, H, W, r, device=dev.index)
            t = _time(lambda: osbf.filter(xx, r, ITERS_, out=out), 5, warmup=2)
            rows.append({"input": tag, "r": r, "kernel": f"tuned ({v})", "depth": d, "depth_run": d,
                         "gpix_iter_s": xx.numel() * ITERS_ / t / 1e9})
            osbf.set_tuned(torch.float32, N * C, H, W, r, 1, "tile", device=dev.index)  # back to the default
        return rows

    small = torch.from_numpy(synth.piecewise_stack(1, 3, 256, 256, seed=52, sigma=0.05)).to(dev)
    return sweep(x, (1, 2, 4, 8, 16), "1x3x4096x4096") + sweep(small, (1, 2, 4), "1x3x256x256")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--depth", type=int, default=0, help="fused passes per launch (0 = library choice)")
    ap.add_argument("--variant", default="auto", choices=["auto", "tile", "strip"],
                    help="float32 single-pass kernel (profiling runs; the default is the library's choice)")
    ap.add_argument("--r", type=int, default=R_)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms (for profiling runs)")
    ap.add_argument("--form", default=None,
                    choices=["fwd_bwd", "batched", "precision", "fast_approximation", "volume_3d", "one_sided_gaussian"],
                    help="run only this form on one GPU and print its JSON (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2108_05021_gb300 import osbf, synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    r = args.r

    x_np = synth.piecewise_stack(N_, C_, H_, W_, seed=rank, sigma=0.05)
    x = torch.from_numpy(x_np).to(dev)
    if args.form is not None:
        one = {"fwd_bwd": lambda: form_fwd_bwd(dev), "batched": lambda: form_batched(dev),
               "precision": lambda: form_precision(dev), "fast_approximation": lambda: form_fast(dev, x),
               "volume_3d": lambda: form_volume(dev), "one_sided_gaussian": lambda: form_gauss(dev, x)}[args.form]
        print(json.dumps({"form": args.form, "result": one()}))
        return
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)

    def step():
        osbf.filter(x, r, ITERS_, depth=args.depth, out=out, variant=args.variant)

    for _ in range(args.warmup):
        step()
    launches_per_step = osbf.last_launch_count(local)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    ms = reduce_max(ev0.elapsed_time(ev1), pg, dev)
    ms_step = ms / args.steps
    pix_iters = N_ * C_ * H_ * W_ * ITERS_
    value = whole_job_rate(pix_iters, ws, ms_step * 1e-3) / 1e6

    # roofline of the forward tile kernel: every launch reads and writes each frame pixel
    # once.  Its average launch duration is measured live with CUDA events on the launching
    # stream: a 30-pass call and a 2-pass call differ by exactly 28 frame-to-frame launches
    # of that kernel (both share the pad launch and the final launch into the output).
    FH, FW = H_ + 2 * r, W_ + 2 * r
    bytes_per_launch = 8.0 * N_ * C_ * FH * FW
    nrep = max(3, min(20, args.steps // 10))

    def timed(iters_):
        for _ in range(2):
            osbf.filter(x, r, iters_, depth=args.depth, out=out, variant=args.variant)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(nrep):
            osbf.filter(x, r, iters_, depth=args.depth, out=out, variant=args.variant)
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / nrep

    if ITERS_ > 2:
        launch_ms = (timed(ITERS_) - timed(2)) / (ITERS_ - 2)
    else:
        launch_ms = ms_step / max(launches_per_step, 1)
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": TRAFFIC_PER_LAUNCH if r == R_ and args.depth in (0, 1) and args.variant != "strip" else None,
                "peak_source": peak_kind, "kernel": "osbf_fwd2 (forward tile kernel, frame to frame, early loads, 32-byte register stores)",
                "bytes_per_launch": bytes_per_launch, "launches_per_step": launches_per_step,
                "launch_ms": launch_ms, "launch_ms_method": "CUDA events: (30-pass call - 2-pass call) / 28",
                "hbm_roofline_equiv_mpix_iter_s": peak * 1e9 / 8.0 / 1e6}

    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_np).pin_memory()
        oh = torch.empty_like(xh).pin_memory()
        for _ in range(2):
            osbf.filter_host(xh, r, ITERS_, out=oh, device=local)
        ne = max(3, min(20, args.steps // 10))
        t0 = time.perf_counter()
        for _ in range(ne):
            osbf.filter_host(xh, r, ITERS_, out=oh, device=local)
        dt = reduce_max((time.perf_counter() - t0) / ne, pg, dev)
        e2e = {"value": whole_job_rate(pix_iters, ws, dt) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(x_np.nbytes), "d2h_bytes_per_step": int(x_np.nbytes),
               "ms_per_step": dt * 1e3, "api": "osbf_filter_host"}

    forms = None
    if rank == 0 and ws == 1 and not args.no_forms:
        forms = {"fwd_bwd": form_fwd_bwd(dev), "batched": form_batched(dev), "precision": form_precision(dev),
                 "fast_approximation": form_fast(dev, x), "volume_3d": form_volume(dev),
                 "one_sided_gaussian": form_gauss(dev, x),
                 "sweep_4096x3_30_passes": form_sweep(dev, x),
                 "plain_mpix_iter_s": value}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, sample, ties = cpu_baseline_sample(x_np[0, 0])
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample, "near_ties": ties}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": N_, "C": C_, "H": H_, "W": W_, "r": r, "iters": ITERS_,
                           "depth": args.depth or "library", "kernel": args.variant if args.variant != "auto" else "library",
                           "l2": "inputs (201 MB) exceed L2; no flush",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary(), "forms": forms}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
