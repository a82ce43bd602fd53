"""Benchmark of the FITrig trigger path on GB300: one JSON line.

A step is one fitrig_detect over a resident synthetic stack: the stack-march
tile statistics, both branches' noise estimates, thresholds, components,
candidates and their sort (every hot-path step).  The default workload is
64 snapshots of 4096 x 4096 FP32 (MeerKAT-like PSF, 500 steady sources, 10
pulsars), window 5, 6 sigma, both branches, median/MAD noise.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank processes its own field (independent
problems, no collective on the data path): weak scaling, max time over ranks.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (the only other place this script runs it).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "snapshot Gpixel/s through tLISI+trigger"
UNIT = "Gpixel/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--noise", choices=["meanstd", "medmad"], default="medmad")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--nsnap", type=int, default=64)
    ap.add_argument("--window", type=int, default=5)
    ap.add_argument("--nsigma", type=float, default=6.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def workload_name(a):
    return (f"{a.nsnap} snapshots of {a.size}x{a.size} {a.storage.upper()} storage, MeerKAT-like "
            f"PSF, both branches, window {a.window}, {a.nsigma:g} sigma, {a.noise} noise")


# ---------------------------------------------------------------- distributed
def dist_init(a):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if a.impl == "ours" else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- peaks / traffic
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def stack_kernel_hash():
    h = hashlib.sha256()
    for f in ("k_stack.cu", "internal.cuh"):
        with open(os.path.join(ROOT, "paper_2509_21754_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(key: str):
    """DRAM bytes per launch of the stack kernel from the committed ncu summary,
    or None when that summary predates the current kernel source."""
    p = os.path.join(ROOT, "profiles", "k_stack_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != stack_kernel_hash():
        return None
    e = d.get("workloads", {}).get(key)
    return None if e is None else float(e["dram_bytes_per_launch"])


# ---------------------------------------------------------------- CPU oracle leg
def oracle_sample(a, stack_np, budget_s=12.0):
    """Time the FP64 oracle (as it stands) on whole-width row strips of the
    workload until about ``budget_s`` of CPU work; returns (Gpx/s, desc, cores)."""
    from oracle import fitrig_oracle as O
    noise = a.noise
    L, ny, nx = stack_np.shape
    rows = 8 * a.window   # 8 tile rows
    done_px, t_used, strips = 0, 0.0, 0
    nstrip = max(1, ny // rows)
    while t_used < budget_s and strips < 4 * nstrip:
        y0 = ((strips * 13) % nstrip) * rows
        strip = stack_np[:, y0:y0 + rows, :]
        t0 = time.perf_counter()
        O.detect(strip, a.window, a.nsigma, O.BRANCH_BOTH, noise)
        t_used += time.perf_counter() - t0
        done_px += L * strip.shape[1] * nx
        strips += 1
    desc = (f"{strips} strips of {L} snapshots x {rows} rows x {nx} columns "
            f"({done_px / 1e6:.0f} Mpixel) of the same stack, FP64 NumPy oracle, "
            f"noise statistics over each strip")
    return done_px / t_used / 1e9, desc, t_used


def reference_arm(a, ws, rank):
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from paper_2509_21754_gb300 import synth
    spec = synth.C2 if a.size == 4096 and a.nsnap == 64 else synth.small_spec(a.nsnap, a.size, a.size)
    stack, _ = synth.make_stack(spec, seed=2026, device="cuda" if _cuda() else "cpu")
    x = stack.cpu().numpy()
    del stack
    from oracle import fitrig_oracle as O
    rows = 40
    per_step = []
    for i in range(a.warmup + a.steps):
        y0 = (i * 7 * rows) % (x.shape[1] - rows)
        strip = x[:, y0:y0 + rows, :]
        t0 = time.perf_counter()
        O.detect(strip, a.window, a.nsigma, O.BRANCH_BOTH, a.noise)
        dt = time.perf_counter() - t0
        if i >= a.warmup:
            per_step.append(dt)
    px = x.shape[0] * rows * x.shape[2]
    t = sum(per_step)
    value = px * a.steps / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(a),
                                        "sample": f"one {rows}-row strip of the stack per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{x.shape[0]} snapshots x {rows} rows x {x.shape[2]} columns per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except ImportError:
        return False


# ---------------------------------------------------------------- our arm
def main():
    a = parse()
    ws, rank = dist_init(a)
    if a.impl == "reference":
        return reference_arm(a, ws, rank)
    import torch

    from paper_2509_21754_gb300 import fitrig as F
    from paper_2509_21754_gb300 import synth

    storage = {"f32": F.F32, "bf16": F.BF16, "f16": F.F16}[a.storage]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.storage]
    noise = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}[a.noise]
    spec = synth.C2 if a.size == 4096 and a.nsnap == 64 else synth.small_spec(a.nsnap, a.size, a.size)
    stack, truth = synth.make_stack(spec, seed=2026 + rank, device="cuda")
    L, ny, nx = stack.shape
    stream = torch.cuda.current_stream()
    plan = F.Plan(nx, ny, L, a.window, a.nsigma, F.BRANCH_BOTH, storage, noise,
                  stream=stream.cuda_stream)
    stack_s = stack.to(tdt)
    plan.push_stack(stack_s)
    torch.cuda.synchronize()

    for _ in range(a.warmup):
        F.fitrig_detect(plan.h)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stack_ms = []
    barrier(ws)
    torch.cuda.synchronize()
    n0 = F.fitrig_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(a.steps):
            rc, ncand = F.fitrig_detect(plan.h)
            stack_ms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_STACK))
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = F.fitrig_launch_count() - n0
    ms = ev0.elapsed_time(ev1) / a.steps
    ms = max_over_ranks(ws, ms)
    px_step = L * ny * nx
    value = ws * px_step / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel (stack march): algorithmic bytes per launch
    Ty, Tx = F.fitrig_tile_grid(plan.h)
    eb = 4 if a.storage == "f32" else 2
    alg_bytes = eb * L * ny * nx + 4 * (L - 2) * Ty * Tx
    k_ms = statistics.mean(stack_ms)
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    traffic_key = f"{a.nsnap}x{a.size}^2/{a.storage}/w{a.window}"
    traffic = measured_traffic(traffic_key)

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not a.no_e2e:
        host = torch.empty((L, ny, nx), dtype=tdt, pin_memory=True)
        host.copy_(stack_s.cpu())
        del stack_s
        host_np = host  # torch CPU tensor, pinned
        tim = []
        ecands = 0
        for i in range(1 + min(a.steps, 5)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F.fitrig_plan_reset(plan.h)
            for k in range(L):
                F.fitrig_push_snapshot(plan.h, host_np[k])
            rc, ncand = F.fitrig_detect(plan.h)
            c = F.fitrig_candidates(plan.h, ncand)
            dt = time.perf_counter() - t0
            if i > 0:
                tim.append(dt)
            ecands = len(c)
        e_ms = 1e3 * statistics.mean(tim)
        e_ms = max_over_ranks(ws, e_ms)
        e2e = {"value": ws * px_step / (e_ms * 1e-3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": eb * L * ny * nx,
               "d2h_bytes_per_step": 32 * ecands + 24, "ms_per_step": e_ms,
               "steps": len(tim)}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu:
        x = stack.to(tdt).float().cpu().numpy()
        v, desc, used = oracle_sample(a, x)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(used, 2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "storage": a.storage,
                       "l2": f"inputs larger than L2 ({eb * L * ny * nx / 1e9:.2f} GB stack)",
                       "candidates": int(ncand), "status": int(rc)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_stack_tile", "kernel_ms": k_ms,
                         "alg_bytes_per_launch": alg_bytes, "peak_kind": peak_kind},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        print(json.dumps(line))
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
