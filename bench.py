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
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-sliding", action="store_true",
                    help="skip the sliding-window leg on the main workload's stack")
    ap.add_argument("--no-spectrum", action="store_true",
                    help="skip the transform-alone leg at power-of-two series lengths")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 256-field batched workload (a few minutes)")
    ap.add_argument("--serving-compression", type=float, default=20.0,
                    help="time compression of the serving leg's Poisson arrivals")
    ap.add_argument("--serving-snapshots", type=int, default=600,
                    help="snapshots each serving field streams (the serving workload's 600)")
    ap.add_argument("--serving-freq", type=int, default=0,
                    help="serving fields also run the real-time frequency branch over their "
                         "last N units")
    ap.add_argument("--paper-run", action="store_true",
                    help="add the paper's end-to-end configuration: 1500 x 4096^2, frequency "
                         "branch with harmonic summing, window 32 (about 110 GB of HBM)")
    ap.add_argument("--no-delta", action="store_true",
                    help="skip the difference-coded half-storage leg on the main workload")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 8 x 50000^2 field with FP32 and BF16 storage (generated and "
                         "pushed one snapshot at a time; about 90 GB of device memory)")
    ap.add_argument("--accumulate", type=int, default=0,
                    help="also time ingest with snapshot accumulation: K raw device "
                         "snapshots summed per stack snapshot (Sec. 3.3.2)")
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
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if a.impl == "ours" else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float, device: str = "cuda") -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, px_per_rank: int, ms_max: float) -> float:
    """Whole-job Gpixel/s: every rank's pixels over the slowest rank's time."""
    return ws * px_per_rank / (ms_max * 1e-3) / 1e9


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


def _oracle_strip(args):
    """Worker of the all-cores oracle leg (a spawned process): one strip."""
    strip, window, nsigma, noise = args
    from oracle import fitrig_oracle as O
    t0 = time.perf_counter()
    O.detect(strip, window, nsigma, O.BRANCH_BOTH, noise)
    return time.perf_counter() - t0


def host_cpu():
    """(logical cores, model name) of the host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_all_cores(a, stack_np, budget_s=12.0):
    """The same oracle on every host core at once: one spawned process per core
    (NumPy single-threaded in each), each taking whole-width strips of the
    stack, for about ``budget_s`` of wall time; returns (Gpx/s, desc, cores)."""
    import multiprocessing as mp
    cores, _ = host_cpu()
    L, ny, nx = stack_np.shape
    rows = 8 * a.window
    nstrip = max(1, ny // rows)
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    ctx = mp.get_context("spawn")   # a fork after CUDA work would hang
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_strip, [(stack_np[:, :rows, :], a.window, a.nsigma, a.noise)] * cores)
        done_px, jobs, t0 = 0, 0, time.perf_counter()
        while time.perf_counter() - t0 < budget_s and jobs < 8 * nstrip:
            batch = []
            for _ in range(cores):
                y0 = ((jobs * 13) % nstrip) * rows
                batch.append((stack_np[:, y0:y0 + rows, :], a.window, a.nsigma, a.noise))
                jobs += 1
            pool.map(_oracle_strip, batch)
            done_px += len(batch) * L * rows * nx
        wall = time.perf_counter() - t0
    desc = (f"{jobs} strips of {L} snapshots x {rows} rows x {nx} columns "
            f"({done_px / 1e6:.0f} Mpixel), {cores} processes, FP64 NumPy oracle")
    return done_px / wall / 1e9, desc, cores


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


# ---------------------------------------------------------------- serving leg
def serving_run(a, F, synth, torch, nfields=32, nsnap=24, compression=20.0, seed=7,
                freq_units=0):
    """C5-like serving: fields stream snapshots (Poisson arrivals, mean 2 s,
    time-compressed) through the server API; returns latency/throughput."""
    import threading
    sides = synth.serving_sides(seed, nfields)
    pools = []
    for k, side in enumerate(sides):
        spec = synth.small_spec(3, side, side)
        st, _ = synth.make_stack(spec, seed=900 + k, device="cuda")
        host = torch.empty((3, side, side), dtype=torch.bfloat16, pin_memory=True)
        host.copy_(st.to(torch.bfloat16))
        pools.append(host)
        del st
    torch.cuda.empty_cache()
    srv = F.fitrig_server_create(150 << 30, 64)
    try:
        ids = []
        for side in sides:
            if freq_units:
                rc, fid = F.fitrig_server_admit_freq(srv, side, side, a.window, a.nsigma, F.BF16,
                                                     F.NOISE_MEDMAD, freq_units)
            else:
                rc, fid = F.fitrig_server_admit(srv, side, side, a.window, a.nsigma, F.BF16,
                                                F.NOISE_MEDMAD)
            ids.append((rc, fid))
        active = [(fid, pools[k]) for k, (rc, fid) in enumerate(ids) if rc == F.OK]
        mean_gap = 2.0 / compression
        t0 = time.monotonic() + 0.2
        pushed = [0]
        lock = threading.Lock()

        def feed(fid, pool, rs):
            t = t0
            for k in range(nsnap):
                t += rs.exponential(mean_gap)
                dt = t - time.monotonic()
                if dt > 0:
                    time.sleep(dt)
                F.fitrig_server_push(srv, fid, pool[k % 3], time.monotonic_ns())
                with lock:
                    pushed[0] += pool.shape[1] * pool.shape[2]

        # results are collected while the fields stream (the records are kept,
        # the candidates counted and dropped, so host memory stays bounded)
        parts, ncand, done = [], [0], threading.Event()

        def collect():
            while True:
                last = done.is_set()
                while True:
                    r, c = F.fitrig_server_poll(srv, cap=1 << 14, cand_cap=1 << 22)
                    if r.size == 0:
                        break
                    parts.append(r)
                    ncand[0] += c.size
                if last:
                    return
                time.sleep(0.05)

        poller = threading.Thread(target=collect)
        poller.start()
        threads = [threading.Thread(target=feed, args=(fid, pool, np.random.default_rng(seed + i)))
                   for i, (fid, pool) in enumerate(active)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        F.fitrig_server_drain(srv)
        t_end = time.monotonic()
        done.set()
        poller.join()
        res = np.concatenate(parts) if parts else np.zeros(0, dtype=F.RESULT_DTYPE)
        ncand = ncand[0]
        lat = (res["t_done_ns"] - res["t_arrival_ns"]) / 1e6
        used, nact, nwait = F.fitrig_server_usage(srv)
        # where the latency went, per unit: the feeder's delay before the push,
        # the host enqueue, the device copy and trigger (GPU timer), and the
        # rest (waiting behind earlier work on the field's stream, callback)
        feeder = (res["t_push_ns"] - res["t_arrival_ns"]) / 1e6
        host = (res["t_enqueued_ns"] - res["t_push_ns"]) / 1e6
        copy = res["copy_ms"].astype(np.float64)
        trig = res["trigger_ms"].astype(np.float64)
        rest = lat - feeder - host - copy - trig
        pct = lambda a: {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)),
                         "max": float(a.max())}
        slow = lat >= np.percentile(lat, 99)
        stages = {"feeder_ms": pct(feeder), "host_enqueue_ms": pct(host), "copy_ms": pct(copy),
                  "trigger_ms": pct(trig), "rest_ms": pct(rest),
                  "slowest_1pct_mean_ms": {k: float(np.mean(a[slow])) for k, a in
                                           (("latency", lat), ("feeder", feeder), ("host", host),
                                            ("copy", copy), ("trigger", trig), ("rest", rest))}}
        return {
            "fields": len(sides), "admitted": len(active), "queued": nwait,
            "snapshots_per_field": nsnap, "units": int(res.size), "candidates": int(ncand),
            "units_truncated": int(np.count_nonzero(res["status"] == F.ETRUNC)),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()),
            "gpx_per_s": pushed[0] / (t_end - t0) / 1e9,
            "compression": compression, "storage": "bf16", "noise": "medmad",
            "reserved_gb": used / 1e9,
            "sides": "uniform 2048..16384, seeded",
            "freq_units": freq_units,
            "stages": stages,
        }
    finally:
        F.fitrig_server_destroy(srv)
        del pools


# ---------------------------------------------------------------- batched leg
def batched_run(a, F, synth, torch, wave_bytes=200e9, reps=3, seed=11):
    """256 fields of uneven size and snapshot count (SKA-AA2-like PSF, BF16
    storage, both branches): resident in waves of <= 200 GB of plan memory,
    each wave one fitrig_batch (one persistent stack march, autotuned CTA
    shape, the whole trigger under one CUDA graph).  Throughput is the pixels
    of all waves over the sum of their median replay times (device time)."""
    fields = synth.batched_fields(seed)
    noise = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}[a.noise]

    def plan_bytes(L, side):   # stack + tile statistics, selection lists, maps
        return 2 * L * side * side * 1.35

    waves, cur, acc = [], [], 0.0
    for k, (L, side) in enumerate(fields):
        b = plan_bytes(L, side)
        if cur and acc + b > wave_bytes:
            waves.append(cur)
            cur, acc = [], 0.0
        cur.append(k)
        acc += b
    if cur:
        waves.append(cur)
    tot_px, tot_ms, t_gen, per_wave = 0, 0.0, 0.0, []
    for wave in waves:
        t0 = time.perf_counter()
        plans = []
        try:
            for k in wave:
                L, side = fields[k]
                p = F.Plan(side, side, L, a.window, a.nsigma, F.BRANCH_BOTH, F.BF16, noise,
                           autotune=True)
                plans.append(p)
                for _, snap in synth.iter_stack(synth.batched_spec(L, side), 5000 + k, "cuda"):
                    F.fitrig_push_snapshot(p.h, snap)   # FP32 in, BF16 on the device
                    del snap
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
            t_gen += time.perf_counter() - t0
            b = F.fitrig_batch_create(plans)
            try:
                F.fitrig_batch_detect(b, len(plans))   # eager run + graph capture
                ms = []
                for _ in range(reps):
                    rc, n = F.fitrig_batch_detect(b, len(plans))
                    ms.append(F.fitrig_batch_ms(b))
            finally:
                F.fitrig_batch_destroy(b)
            px = sum(fields[k][0] * fields[k][1] ** 2 for k in wave)
            wms = statistics.median(ms)
            tot_px += px
            tot_ms += wms
            per_wave.append({"fields": len(wave), "gpixel": px / 1e9, "ms": wms,
                             "candidates": int(np.sum(n)), "status": int(rc)})
        finally:
            for p in plans:
                p.close()
            torch.cuda.empty_cache()
    return {"workload": "256 fields, side U{1024..8192}, U{16..128} snapshots, SKA-AA2-like PSF, "
                        f"BF16 storage, both branches, window {a.window}, {a.nsigma:g} sigma, "
                        f"{a.noise} noise", "waves": len(waves), "gpixel": tot_px / 1e9,
            "ms": tot_ms, "value": tot_px / (tot_ms * 1e-3) / 1e9, "unit": UNIT,
            "timing": f"median of {reps} graph replays per wave, CUDA events",
            "generation_s": round(t_gen, 1), "per_wave": per_wave}


# ---------------------------------------------------------------- large-field leg
def large_run(a, F, synth, torch, storage, steps=5, seed=3030):
    """C3: 8 snapshots of 50000 x 50000 (MeerKAT-like PSF, 10^4 steady sources,
    50 pulsars), both branches, window 5, 6 sigma; snapshots generated on the
    device one at a time and pushed (FP32 in, stored in the chosen type)."""
    spec = synth.C3
    noise = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}[a.noise]
    st = torch.cuda.current_stream()
    plan = F.Plan(spec.nx, spec.ny, spec.nsnap, 5, 6.0, F.BRANCH_BOTH, storage, noise,
                  stream=st.cuda_stream)
    try:
        for _, snap in synth.iter_stack(spec, seed, "cuda"):
            F.fitrig_push_snapshot(plan.h, snap)
            del snap
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        F.fitrig_detect(plan.h)
        F.fitrig_detect(plan.h)
        ms, stack_ms = [], []
        for _ in range(steps):
            rc, n = F.fitrig_detect(plan.h)
            ms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_DETECT))
            stack_ms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_STACK))
        Ty, Tx = F.fitrig_tile_grid(plan.h)
    finally:
        plan.close()
    L, px = spec.nsnap, spec.ny * spec.nx
    eb = 4 if storage == F.F32 else 2
    t, ts = statistics.median(ms), statistics.median(stack_ms)
    alg = eb * L * px + 5 * (L - 2) * Ty * Tx
    peak, _ = hbm_peak()
    return {"workload": "8 snapshots of 50000x50000, MeerKAT-like PSF, both branches, window 5, "
                        f"6 sigma, {a.noise} noise", "storage": {F.F32: "f32", F.BF16: "bf16",
                                                                F.F16: "f16"}[storage],
            "detect_ms": t, "value": L * px / (t * 1e-3) / 1e9, "unit": UNIT,
            "stack_ms": ts, "stack_frac_of_hbm": alg / (ts * 1e-3) / 1e9 / peak,
            "candidates": int(n), "status": int(rc)}


# ---------------------------------------------------------------- the paper's end-to-end run
PAPER_H100_S = 6.34   # Sec. 3 (real-data evaluation): 1500 snapshots of 4096^2, image loading to pulsar position


def paper_run(a, F, synth, torch, steps=3, seed=4040, ring=64):
    """The configuration of the paper's end-to-end timing (the real-data evaluation of Sec. 3): 1500
    snapshots of 4096 x 4096 (MeerKAT-like PSF, the 64-snapshot workload's
    source rules), image-frequency branch with harmonic summing (m_max = 8),
    window 32, 6 sigma, mean/std noise, FP32.  Device leg: detects over the
    resident stack (median of `steps`).  End-to-end leg: every snapshot pushed
    from pinned host memory (a ring of `ring` distinct snapshots reused in
    order, so the series repeats with period `ring`), the detect and the
    candidate read-back, wall clock."""
    import dataclasses
    spec = dataclasses.replace(synth.C2, nsnap=1500)
    L, ny, nx = spec.nsnap, spec.ny, spec.nx
    st = torch.cuda.current_stream()
    plan = F.Plan(nx, ny, L, 32, 6.0, F.BRANCH_FREQ, F.F32, F.NOISE_MEANSTD,
                  stream=st.cuda_stream, harmonics=8)
    host = torch.empty((ring, ny, nx), dtype=torch.float32, pin_memory=True)
    try:
        t0 = time.perf_counter()
        for k, snap in synth.iter_stack(spec, seed, "cuda"):
            F.fitrig_push_snapshot(plan.h, snap)
            if k < ring:
                host[k].copy_(snap)
            del snap
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        torch.cuda.empty_cache()
        F.fitrig_detect(plan.h)
        F.fitrig_detect(plan.h)
        ms, stages = [], []
        for _ in range(steps):
            rc, n = F.fitrig_detect(plan.h)
            ms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_DETECT))
            stages.append({"stack": F.fitrig_kernel_ms(plan.h, F.KERNEL_STACK),
                           "spectrum": F.fitrig_kernel_ms(plan.h, F.KERNEL_SPECTRUM)})
        e2e, cbuf, craw = [], None, None
        for i in range(1 + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F.fitrig_plan_reset(plan.h)
            done = 0
            while done < L:
                c = min(ring, L - done)
                F.fitrig_push_snapshots(plan.h, host[:c])
                done += c
            rc2, n2 = F.fitrig_detect(plan.h)
            if cbuf is None or len(cbuf) < n2:
                craw = torch.empty(max(n2, 1) * F.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8,
                                   pin_memory=True)
                cbuf = craw.numpy().view(F.CANDIDATE_DTYPE)
            F.fitrig_candidates(plan.h, n2, out=cbuf)
            if i > 0:
                e2e.append(time.perf_counter() - t0)
        del cbuf, craw
    finally:
        plan.close()
        del host
    px = L * ny * nx
    t = statistics.median(ms)
    e_s = statistics.median(e2e)
    return {"workload": "1500 snapshots of 4096x4096 FP32, MeerKAT-like PSF, image-frequency "
                        "branch, harmonic sum m_max 8, window 32, 6 sigma, meanstd noise",
            "detect_ms": t, "value": px / (t * 1e-3) / 1e9, "unit": UNIT,
            "stages_ms": {k: statistics.median(s[k] for s in stages) for k in stages[0]},
            "e2e_s": e_s, "e2e_value": px / e_s / 1e9,
            "e2e_note": f"pushes from pinned host memory ({ring} distinct snapshots reused in "
                        "order), detect and candidate read-back; the paper's time also loads "
                        "the images from storage",
            "h2d_bytes_per_step": 4 * px, "paper_h100_s": PAPER_H100_S,
            "candidates": int(n), "status": int(rc), "generation_s": round(gen_s, 1)}


# ---------------------------------------------------------------- spectrum leg
def spectrum_run(F, torch, T=16384, lengths=(256, 512, 1024, 2048, 4096), reps=5):
    """The image-frequency transform alone at the paper's power-of-two series
    lengths (L - 2 = 2^m), on T = 16384 series (a 4096^2 image at window 32):
    the radix FFT against the direct O(n^2) warp kernel on the same cube.
    Bytes per launch = the cube read once (4 n T) + eta and bin written (8 T)."""
    out = {"tiles": T, "timing": f"median of {reps} launches, CUDA events", "lengths": {}}
    g = torch.Generator(device="cuda").manual_seed(5)
    for n in lengths:
        x = torch.randn(n, T, device="cuda", generator=g).abs_().square_().add_(0.5)
        eta = torch.empty(T, device="cuda")
        kb = torch.empty(T, dtype=torch.int32, device="cuda")
        row = {}
        for name, m in (("radix", F.SPECTRUM_RADIX), ("direct", F.SPECTRUM_DIRECT)):
            F.fitrig_spectrum_map(x, n, T, T, 1, eta, kb, m)
            ms = statistics.median(F.fitrig_spectrum_map(x, n, T, T, 1, eta, kb, m)
                                   for _ in range(reps))
            row[f"{name}_ms"] = ms
            row[f"{name}_gb_per_s"] = (4 * n * T + 8 * T) / (ms * 1e-3) / 1e9
        row["speedup"] = row["direct_ms"] / row["radix_ms"]
        out["lengths"][str(n)] = row
        del x, eta, kb
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- sliding-window leg
def sliding_run(a, F, torch, stack, storage, reps=5):
    """The sliding-window mode (the odd w x w window centred on every pixel) on
    the main workload's stack: the detect and its march (k_slide).  Bytes of
    the march per launch: the stack read once (b L px) and v written per pixel
    and unit (4 (L - 2) px)."""
    L, ny, nx = stack.shape
    eb = 4 if a.storage == "f32" else 2
    st = torch.cuda.current_stream()
    plan = F.Plan(nx, ny, L, a.window, a.nsigma, F.BRANCH_IMAGE, storage,
                  {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}[a.noise],
                  stream=st.cuda_stream, stride=F.STRIDE_SLIDING)
    try:
        plan.push_stack(stack)
        torch.cuda.synchronize()
        F.fitrig_detect(plan.h)
        F.fitrig_detect(plan.h)
        ms, mms = [], []
        for _ in range(reps):
            rc, n = F.fitrig_detect(plan.h)
            ms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_DETECT))
            mms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_STACK))
    finally:
        plan.close()
    px = L * ny * nx
    t, tm = statistics.median(ms), statistics.median(mms)
    alg = eb * px + 4 * (L - 2) * ny * nx
    peak, kind = hbm_peak()
    return {"workload": f"{L} snapshots of {nx}x{ny}, sliding {a.window}x{a.window} window, image "
                        f"branch, {a.nsigma:g} sigma, {a.noise} noise",
            "detect_ms": t, "value": px / (t * 1e-3) / 1e9, "unit": UNIT, "march_ms": tm,
            "march_gb_per_s": alg / (tm * 1e-3) / 1e9, "march_frac_of_hbm": alg / (tm * 1e-3) / 1e9 / peak,
            "candidates": int(n), "status": int(rc)}


# ---------------------------------------------------------------- difference-coded half storage
class _DevArr:
    """A borrowed device buffer seen through the CUDA array interface."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape,
                                         "typestr": typestr, "version": 2, "strides": None}


def delta_run(a, F, torch, stack, steps=20, e2e_steps=5):
    """The main workload with difference-coded half storage (FP32 key frame,
    BF16 or FP16 differences; FITRIG_OPT_CODING): device detect over the
    resident stack, its march against the algorithmic bytes (key 4 B/px once,
    differences 2 B/px per later snapshot, v and arg-max per tile and unit),
    and for BF16 end to end from pinned host buffers that already hold the
    coded form (the key frame as FP32, the differences as BF16: a producer
    that runs the same coder), with the candidates read back every step."""
    L, ny, nx = stack.shape
    st = torch.cuda.current_stream()
    noise = {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}[a.noise]
    peak, kind = hbm_peak()
    out = {"workload": workload_name(a).replace(f"{a.storage.upper()} storage",
                                                "difference-coded storage"),
           "timing": f"CUDA events around {steps} detects"}
    for name, code, tdt in (("bf16", F.BF16, torch.bfloat16), ("f16", F.F16, torch.float16)):
        plan = F.Plan(nx, ny, L, a.window, a.nsigma, F.BRANCH_BOTH, code, noise,
                      stream=st.cuda_stream, coding=F.CODING_DELTA)
        try:
            plan.push_stack(stack)           # FP32 on the device, coded there
            torch.cuda.synchronize()
            for _ in range(3):
                F.fitrig_detect(plan.h)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sms = []
            e0.record(st)
            for _ in range(steps):
                rc, n = F.fitrig_detect(plan.h)
                sms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_STACK))
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            Ty, Tx = F.fitrig_tile_grid(plan.h)
            alg = 4 * ny * nx + 2 * (L - 1) * ny * nx + (4 + (1 if a.window <= 6 else 0)) * (L - 2) * Ty * Tx
            k_ms = statistics.mean(sms)
            leg = {"detect_ms": ms, "value": L * ny * nx / (ms * 1e-3) / 1e9, "unit": UNIT,
                   "march_ms": k_ms, "march_alg_bytes": alg,
                   "march_frac_of_hbm": alg / (k_ms * 1e-3) / 1e9 / peak,
                   "candidates": int(n), "status": int(rc)}
            if name == "bf16" and not a.no_e2e:
                # the coded form as a producer would send it, read back once
                key = torch.empty((ny, nx), dtype=torch.float32, pin_memory=True)
                qh = torch.empty((L - 1, ny, nx), dtype=tdt, pin_memory=True)
                for s_ in range(L):
                    ptr, pitch = F.fitrig_stack_device_ptr(plan.h, s_)
                    view = torch.as_tensor(_DevArr(ptr, (ny, pitch), "<f4" if s_ == 0 else "<i2"),
                                           device="cuda")
                    if s_ == 0:
                        key.copy_(view[:, :nx])
                    else:
                        qh[s_ - 1].copy_(view[:, :nx].view(tdt))
                torch.cuda.synchronize()
                tim, cbuf, ecands = [], None, 0
                for i in range(1 + e2e_steps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    F.fitrig_plan_reset(plan.h)
                    F.fitrig_push_snapshot(plan.h, key)
                    F.fitrig_push_snapshots(plan.h, qh)
                    rc2, n2 = F.fitrig_detect(plan.h)
                    if cbuf is None or len(cbuf) < n2:
                        craw = torch.empty(max(n2, 1) * F.CANDIDATE_DTYPE.itemsize,
                                           dtype=torch.uint8, pin_memory=True)
                        cbuf = craw.numpy().view(F.CANDIDATE_DTYPE)
                    c = F.fitrig_candidates(plan.h, n2, out=cbuf)
                    dt = time.perf_counter() - t0
                    if i > 0:
                        tim.append(dt)
                    ecands = len(c)
                e_ms = 1e3 * statistics.mean(tim)
                leg["e2e"] = {"value": L * ny * nx / (e_ms * 1e-3) / 1e9, "unit": UNIT,
                              "h2d_bytes_per_step": 4 * ny * nx + 2 * (L - 1) * ny * nx,
                              "d2h_bytes_per_step": 32 * ecands + 24, "ms_per_step": e_ms,
                              "steps": len(tim), "candidates": int(n2)}
                del key, qh, cbuf
            out[name] = leg
        finally:
            plan.close()
    return out


# ---------------------------------------------------------------- accumulation leg
def accumulate_run(a, F, torch, stack, storage, reps=3):
    """Ingest with snapshot accumulation (Sec. 3.3.2): K raw device snapshots
    (the stack's snapshots, cycled) pushed per stack snapshot, then a detect.
    Bytes per raw push: read the raw snapshot, read and write the FP32 sum
    (the first push of a block only writes it, the last writes the stack)."""
    K = a.accumulate
    L, ny, nx = stack.shape
    eb = 4 if a.storage == "f32" else 2
    st = torch.cuda.current_stream()
    plan = F.Plan(nx, ny, L, a.window, a.nsigma, F.BRANCH_BOTH, storage,
                  {"meanstd": F.NOISE_MEANSTD, "medmad": F.NOISE_MEDMAD}[a.noise],
                  stream=st.cuda_stream, accumulate=K)
    try:
        ms = []
        for rep in range(reps + 1):
            F.fitrig_plan_reset(plan.h)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for r in range(L * K):
                F.fitrig_push_snapshot(plan.h, stack[r % L])
            e1.record(st)
            torch.cuda.synchronize()
            if rep:
                ms.append(e0.elapsed_time(e1))
        rc, n = F.fitrig_detect(plan.h)
    finally:
        plan.close()
    px = ny * nx
    nbytes = L * px * (12 * K - 8 + eb)   # per block: 8 + 12 (K - 2) + (8 + eb) B/px
    t = statistics.median(ms)
    return {"k": K, "raw_snapshots": L * K, "ms": t, "raw_gpixel_per_s": L * K * px / (t * 1e-3) / 1e9,
            "gb_per_s": nbytes / (t * 1e-3) / 1e9,
            "bytes": "raw 4 B/px read per push; FP32 sum read and written between pushes; "
                     "stack written once per block", "detect_status": int(rc),
            "candidates": int(n)}


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
    groups = {"stack": F.KERNEL_STACK, "noise": F.KERNEL_NOISE, "select": F.KERNEL_SELECT,
              "spectrum": F.KERNEL_SPECTRUM, "detect": F.KERNEL_DETECT}
    group_ms = {k: [] for k in groups}
    barrier(ws)
    torch.cuda.synchronize()
    n0 = F.fitrig_launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(a.steps):
            rc, ncand = F.fitrig_detect(plan.h)
            stack_ms.append(F.fitrig_kernel_ms(plan.h, F.KERNEL_STACK))
            for k, g in groups.items():
                group_ms[k].append(F.fitrig_kernel_ms(plan.h, g))
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = F.fitrig_launch_count() - n0
    ms = ev0.elapsed_time(ev1) / a.steps
    ms = max_over_ranks(ws, ms)
    px_step = L * ny * nx
    value = job_throughput(ws, px_step, ms)

    # roofline of the dominant kernel (stack march): algorithmic bytes per launch
    Ty, Tx = F.fitrig_tile_grid(plan.h)
    eb = 4 if a.storage == "f32" else 2
    # one read of every stored pixel, one v write per tile per unit, and the
    # in-tile arg-max byte the thread-per-tile march (window <= 6) writes
    out_b = 4 + (1 if a.window <= 6 else 0)
    alg_bytes = eb * L * ny * nx + out_b * (L - 2) * Ty * Tx
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
        host_np = host  # torch CPU tensor, pinned
        tim = []
        ecands = 0
        # candidates land in a reused pinned buffer (grown when a detect needs more)
        cbuf = None
        for i in range(1 + min(a.steps, 5)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F.fitrig_plan_reset(plan.h)
            F.fitrig_push_snapshots(plan.h, host_np)
            rc, ncand = F.fitrig_detect(plan.h)
            if cbuf is None or len(cbuf) < ncand:
                craw = torch.empty(max(ncand, 1) * F.CANDIDATE_DTYPE.itemsize, dtype=torch.uint8,
                                   pin_memory=True)
                cbuf = craw.numpy().view(F.CANDIDATE_DTYPE)
            c = F.fitrig_candidates(plan.h, ncand, out=cbuf)
            dt = time.perf_counter() - t0
            if i > 0:
                tim.append(dt)
            ecands = len(c)
        del host, host_np, cbuf
        e_ms = 1e3 * statistics.mean(tim)
        e_ms = max_over_ranks(ws, e_ms)
        e2e = {"value": job_throughput(ws, px_step, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": eb * L * ny * nx,
               "d2h_bytes_per_step": 32 * ecands + 24, "ms_per_step": e_ms,
               "steps": len(tim)}

    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu:
        x = stack.to(tdt).float().cpu().numpy()
        v1, desc1, used = oracle_sample(a, x)
        vall, descall, cores = oracle_all_cores(a, x)
        _, model = host_cpu()
        cpu = {"value": vall, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": descall,
               "single_core": {"value": v1, "cores": 1, "sample": desc1, "seconds": round(used, 2)},
               "host_cpu": model}

    accum = large = spectrum = None
    if rank == 0 and ws == 1 and a.accumulate > 1:
        accum = accumulate_run(a, F, torch, stack, storage)
    if rank == 0 and ws == 1 and not a.no_spectrum:
        spectrum = spectrum_run(F, torch)
    sliding = None
    if rank == 0 and ws == 1 and not a.no_sliding:
        sliding = sliding_run(a, F, torch, stack_s, storage)
    delta = None
    if rank == 0 and ws == 1 and not a.no_delta:
        delta = delta_run(a, F, torch, stack)

    serving = batched = None
    legs = rank == 0 and ws == 1 and (not a.no_large or a.paper_run or not a.no_serving or
                                      not a.no_batched)
    if legs:   # the remaining legs need the device memory of the main workload
        plan.close()
        del stack, stack_s
        torch.cuda.empty_cache()
    paper = None
    if rank == 0 and ws == 1 and a.paper_run:
        paper = paper_run(a, F, synth, torch)
    if rank == 0 and ws == 1 and not a.no_large:
        large = {"f32": large_run(a, F, synth, torch, F.F32),
                 "bf16": large_run(a, F, synth, torch, F.BF16)}
    if rank == 0 and ws == 1 and not a.no_serving:
        serving = serving_run(a, F, synth, torch, freq_units=a.serving_freq,
                              compression=a.serving_compression, nsnap=a.serving_snapshots)
    if rank == 0 and ws == 1 and not a.no_batched:
        batched = batched_run(a, F, synth, torch)

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
                         "kernel": "k_stack_small" if a.window <= 6 else "k_stack_tile",
                         "kernel_ms": k_ms, "alg_bytes_per_launch": alg_bytes,
                         "peak_kind": peak_kind},
            "stages_ms": {k: statistics.mean(v) for k, v in group_ms.items()},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "serving": serving,
            "batched": batched,
            "accumulate": accum,
            "spectrum_pow2": spectrum,
            "sliding": sliding,
            "delta": delta,
            "large": large,
            "paper_run": paper,
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        print(json.dumps(line))
    if plan.h is not None:
        plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
