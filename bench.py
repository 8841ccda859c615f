"""Benchmark of the multi-level 2-D DWT on GB300 (one JSON line on stdout).

Workload (one step): an 8192 x 8192 float32 synthetic textured image
(uniform 0..255 plus four random sinusoids of amplitude 16), CDF 9/7,
6 levels, forward transform then inverse transform, scheme Monolithic*
(the paper's best), through the library's C ABI.  Metric: Gpixel/s = image
pixels transformed (2 x 8192^2 per step: forward and inverse) per second.
Inputs (268 MB per buffer) are larger than L2 (129 MB), so no L2 flush is
needed between steps.

``--impl reference`` times the oracle (plain C, FP64) on the host cores on a
bounded sample of the same workload (a 1024^2 image per step).

Multi-GPU: the transform of one image does not shard, so N GPUs run N
independent replicas (weak scaling); value = pixels of all ranks / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpixel/s per 2-D DWT (forward + inverse, 6 levels)"
UNIT = "Gpixel/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=8192)
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--wavelet", default="cdf97", choices=["cdf53", "cdf97"])
    ap.add_argument("--scheme", default="monolithic*")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload_name(a):
    return (f"{a.size}x{a.size} float32 textured image, CDF {'9/7' if a.wavelet == 'cdf97' else '5/3'}, "
            f"{a.levels} levels, forward + inverse, scheme {a.scheme}")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1605_00561_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = [(t, l.split(", ")) for t, l in self.lines if l.count(",") >= 8]
        inside = [r for t, r in rows if self.t0 and self.t1 and self.t0 <= t <= self.t1] or [r for _, r in rows]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def cpu_baseline_oracle(a, n=None):
    """The oracle as it stands (single-threaded C, FP64) on host cores."""
    import numpy as np

    import oracle
    from paper_1605_00561_gb300 import inputs
    n = n or a.size
    oid = oracle.CDF97 if a.wavelet == "cdf97" else oracle.CDF53
    x = inputs.textured_image(n, n, seed=2).astype(np.float64)
    t = time.perf_counter()
    c = oracle.dwt2(x, oid, a.levels)
    oracle.dwt2(c, oid, a.levels, inverse=True)
    dt = time.perf_counter() - t
    return 2.0 * n * n / dt / 1e9, dt, n


def run_reference(a, rank, world):
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1605_00561_gb300 import inputs
    n = 1024
    oid = oracle.CDF97 if a.wavelet == "cdf97" else oracle.CDF53
    x = inputs.textured_image(n, n, seed=2).astype(np.float64)
    for _ in range(a.warmup):
        oracle.dwt2(oracle.dwt2(x, oid, a.levels), oid, a.levels, inverse=True)
    t = time.perf_counter()
    for _ in range(a.steps):
        oracle.dwt2(oracle.dwt2(x, oid, a.levels), oid, a.levels, inverse=True)
    dt = time.perf_counter() - t
    value = 2.0 * n * n * a.steps / dt / 1e9
    sample = f"{n}x{n} per step (same textured recipe, CDF, levels, fwd+inv), FP64 C oracle, 1 thread"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3 / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_1605_00561_gb300 import dwt, inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    n, L = a.size, a.levels
    x = torch.from_numpy(inputs.textured_image(n, n, seed=2 + rank)).cuda()
    c = torch.empty_like(x)
    y = torch.empty_like(x)
    plan = dwt.Plan(n, n, a.wavelet, L, "f32", scheme=a.scheme)
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    pitch = n * 4

    def step():
        dwt.dwt2_forward(plan.handle, x.data_ptr(), pitch, c.data_ptr(), pitch, sid)
        dwt.dwt2_inverse(plan.handle, c.data_ptr(), pitch, y.data_ptr(), pitch, sid)

    for _ in range(max(a.warmup, 3)):
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(local)
    gpu_id = str(getattr(props, "uuid", local))
    gpu_id = gpu_id if gpu_id.startswith("GPU-") else f"GPU-{gpu_id}" if len(gpu_id) > 30 else str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    sampler.mark("t0")
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark("t1")
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / a.steps
    value = world * 2.0 * n * n * a.steps / (ms / 1e3) / 1e9
    assert dwt.dwt_plan_device_status(plan.handle) == dwt.DWT_OK

    # Per-kernel durations: the same K steps again with CUDA events around
    # every launch on the launching stream.  Events serialise the launches
    # (no programmatic overlap), so this pass is kept out of the timed region.
    dwt.dwt_plan_read_profile(plan.handle)
    dwt.dwt_plan_set_profiling(plan.handle, True)
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    prof = dwt.dwt_plan_read_profile(plan.handle)
    dwt.dwt_plan_set_profiling(plan.handle, False)

    # dominant kernel: largest share of the profiled time
    top = max(prof, key=lambda p: p["total_ms"])
    per_launch_s = top["total_ms"] / top["launches"] / 1e3
    bytes_per_launch = top["algorithmic_bytes"] / top["launches"]
    achieved = bytes_per_launch / per_launch_s / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        entry = tr.get(f"{a.wavelet}/{a.scheme}/{n}/L{L}/{top['name']}")
        if entry and entry.get("kernel_hash") == kernel_source_hash():
            traffic = entry["bytes_per_launch"]
    except (OSError, ValueError):
        pass
    total_prof = sum(p["total_ms"] for p in prof)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": top["name"],
                "share": top["total_ms"] / total_prof if total_prof else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s",
                "timing": "CUDA events around each launch, profiled pass of the same steps after the timed region"}
    per_kernel = {p["name"]: round(p["total_ms"] / p["launches"] * 1e3, 2) for p in prof}

    # end to end through the host-buffer entry points
    xh = x.cpu().pin_memory()
    ch = torch.empty_like(xh).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    dwt.dwt2_forward_host(plan.handle, xh.data_ptr(), pitch, ch.data_ptr(), pitch, sid)
    dwt.dwt2_inverse_host(plan.handle, ch.data_ptr(), pitch, yh.data_ptr(), pitch, sid)
    torch.cuda.synchronize()
    barrier()
    k2 = max(1, a.e2e_steps)
    e0.record(stream)
    for _ in range(k2):
        dwt.dwt2_forward_host(plan.handle, xh.data_ptr(), pitch, ch.data_ptr(), pitch, sid)
        dwt.dwt2_inverse_host(plan.handle, ch.data_ptr(), pitch, yh.data_ptr(), pitch, sid)
    e1.record(stream)
    torch.cuda.synchronize()
    ms2 = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms2], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms2 = float(t.item())
    e2e = {"value": world * 2.0 * n * n * k2 / (ms2 / 1e3) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 2 * n * n * 4, "d2h_bytes_per_step": 2 * n * n * 4}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, dt, nn = cpu_baseline_oracle(a)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nn}x{nn} forward + inverse once ({dt:.1f} s), FP64 C oracle, 1 thread"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "image": f"{n}x{n}", "levels": L, "wavelet": a.wavelet,
                       "scheme": a.scheme, "l2": "inputs (268 MB per buffer) larger than L2, no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "per_launch_us": per_kernel, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks, "gpu_launches": 2 * L * a.steps,
        }), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
