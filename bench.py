"""Throughput benchmark of the One-Sided Box Filter library on GB300.

Workload: the plain float32 forward on 1 x 3 x 4096 x 4096 synthetic piecewise-constant
+ noise images (40 rectangles, 20 triangles, sigma 0.05, each channel its own plane),
r = 8, 30 passes.  A "step" is one full filter call (all 30 passes) on that batch.
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
  cpu_baseline the CPU oracle on the host cores, on a bounded sample (one 1024 x 1024
               crop of the same image, r = 8) -- a reported baseline, not the target.

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


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
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
        for l in getattr(self, "lines", []):
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
    for about `seconds_hint` seconds of work.  Returns (Mpixel*iter/s, cores, description)."""
    import oracle

    crop = np.ascontiguousarray(x_plane[:1024, :1024], dtype=np.float64)
    t0 = time.perf_counter()
    oracle.filter(crop, R_, 1)
    t1 = time.perf_counter() - t0
    iters = max(1, min(ITERS_, int(seconds_hint / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.filter(crop, R_, iters)
    dt = time.perf_counter() - t0
    mpx = crop.size * iters / dt / 1e6
    return mpx, oracle.threads(), f"1 plane, 1024x1024 crop of channel 0, r={R_}, {iters} passes, FP64 direct sums"


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--depth", type=int, default=0, help="fused passes per launch (0 = library choice)")
    ap.add_argument("--r", type=int, default=R_)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
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
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)

    def step():
        osbf.filter(x, r, ITERS_, depth=args.depth, out=out)

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
    ms = ev0.elapsed_time(ev1)
    if pg:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    pix_iters = N_ * C_ * H_ * W_ * ITERS_
    value = ws * pix_iters / (ms_step * 1e-3) / 1e6

    # roofline of the forward tile kernel: every launch reads and writes each frame pixel once
    FH, FW = H_ + 2 * r, W_ + 2 * r
    bytes_per_launch = 8.0 * N_ * C_ * FH * FW
    launch_ms = ms_step / max(launches_per_step, 1)
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_source": peak_kind, "kernel": "osbf_fwd_tile",
                "bytes_per_launch": bytes_per_launch, "launches_per_step": launches_per_step}

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
        dt = (time.perf_counter() - t0) / ne
        if pg:
            t = torch.tensor([dt], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": ws * pix_iters / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(x_np.nbytes),
               "d2h_bytes_per_step": int(x_np.nbytes), "ms_per_step": dt * 1e3, "api": "osbf_filter_host"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, sample = cpu_baseline_sample(x_np[0, 0])
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": N_, "C": C_, "H": H_, "W": W_, "r": r, "iters": ITERS_,
                           "depth": args.depth or "library", "l2": "inputs (201 MB) exceed L2; no flush",
                           "parallelism": f"replicas x{ws}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
