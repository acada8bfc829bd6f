"""Benchmark: full FMM data-structure rebuild throughput (Mpoints/s).

Workload (one "step"): one fmm_build of N = M = 2^24 float32 points drawn
i.i.d. uniform in the unit cube (sources and receivers independent), L = 7:
Morton keys, sort, boxes of levels 0..7, E2 and E4 lists of levels 2..7.
Inputs (402 MB) are larger than L2, so no flush is needed between steps.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the CPU oracle
instead, on bounded samples of the same workload (see ``reference_arm``).
Multi-GPU (torchrun): every rank builds its own replica (the path has no
exchange step); value = all points of all ranks / max-over-ranks time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpts/s full FMM-structure rebuild at N=M=2^24 L=7; batched vs plain; p99 ms"
N_PTS = 1 << 24
LEVEL = 7
SEEDS = (3, 4)
WORKLOAD = "plain build N=M=2^24 uniform [0,1)^3 float32, L=7, lists at levels 2..7"

# Readback of one build: status word + box counts (first read) and status
# word + list totals (second read), see api.cu.
D2H_BYTES = 16 + 2 * (2 * 22 * 4) + 16 + 22 * 2 * 8


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    INTERVAL_MS = 50

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        """Starts sampling and returns once nvidia-smi delivers samples, so
        that the timed region that follows is covered from its start."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0:
            time.sleep(0.01)
        self.first = len(self.lines)  # samples from here on fall in the timed region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the samples taken during the timed region (else the last one before it)
        during = self.lines[self.first:] or self.lines[-1:]
        for ln in during:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, dist, device: str = "cuda") -> float:
    """The slowest rank's time (replicas: the job ends when the last one does)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, ms: float, world: int) -> float:
    """Whole-job throughput in units per second: every rank's units over the
    max-over-ranks time."""
    return units_per_rank * world / (ms / 1e3)


def _algorithmic_bytes(tree) -> dict:
    """Compulsory traffic of one build: inputs read once, outputs written once."""
    n, m = tree.src.n, tree.recv.n
    b = {"xyz": 12 * (n + m), "perm": 4 * (n + m), "boxes": 0, "e2": 0, "e4": 0}
    for sd in (tree.src, tree.recv):
        for l in range(tree.L + 1):
            nb = sd.nbox[l]
            b["boxes"] += 8 * nb + 4 * (nb + 1) + 4 * nb
    for l in range(2, tree.L + 1):
        nr = tree.recv.nbox[l]
        b["e2"] += 4 * (nr + 1) + 4 * tree.nnz_e2[l]
        b["e4"] += 4 * (nr + 1) + 4 * tree.nnz_e4[l]
    b["total"] = sum(v for k, v in b.items())
    return b


def _src_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1301_1704_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic_record() -> dict:
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    try:
        return json.load(open(p))
    except ValueError:
        return {}


def _build_traffic(workload: str):
    """ncu DRAM bytes (read + write) of all kernels of one build of
    `workload`, if they were captured from the current sources."""
    e = _traffic_record().get(workload)
    if not e or e.get("src_hash") != _src_hash():
        return None
    return e.get("dram_bytes_per_build")


def cpu_baseline() -> dict:
    """The oracle on the whole benchmark workload (config 2): its OpenMP
    build on all host cores (about 3 s on 16 Grace cores), and the plain build
    on one core (about 25 s)."""
    from oracle import oracle
    from paper_1301_1704_gb300 import workloads
    src = workloads.uniform(N_PTS, SEEDS[0])
    recv = workloads.uniform(N_PTS, SEEDS[1])
    pts = len(src) + len(recv)
    out = {}
    for parallel in (True, False):
        oracle.build(parallel=parallel)
        out[parallel] = oracle.time_build(src, recv, L=LEVEL, mode=oracle.MODE_STENCIL,
                                          parallel=parallel)
    cores = os.cpu_count() or 1
    return {"value": pts / out[True] / 1e6, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
            "sample": f"the whole benchmark workload ({len(src)} src + {len(recv)} recv), L={LEVEL},"
                      f" stencil lists; the oracle's OpenMP build on {cores} threads:"
                      f" {out[True]:.2f} s",
            "single_thread": {"value": pts / out[False] / 1e6, "cores": 1,
                              "seconds": out[False]}}


def reference_arm(args) -> None:
    """`--impl reference`: the CPU oracle (its OpenMP build, all host cores)
    on the benchmark's own workload, one whole config-2 build (2^24 + 2^24
    points, L = 7, every list) per step -- about 3 s a step on 16 Grace
    cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle
    from paper_1301_1704_gb300 import workloads
    oracle.build(parallel=True)
    cores = os.cpu_count() or 1
    npts = args.points
    src = workloads.uniform(npts, SEEDS[0])
    recv = workloads.uniform(npts, SEEDS[1])
    times = []
    for step in range(args.warmup + args.steps):
        dt = oracle.time_build(src, recv, L=args.level, mode=oracle.MODE_STENCIL, parallel=True)
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    val = 2 * npts * len(times) / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD if (npts, args.level) == (N_PTS, LEVEL) else
                   f"N=M={npts} uniform, L={args.level}", "N": npts, "M": npts, "L": args.level,
                   "seeds": list(SEEDS)},
        "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step one whole build of the workload; the oracle's "
                                   f"OpenMP build on {cores} threads"},
        "e2e": {"value": val, "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _pct(ms, q):
    ms = sorted(ms)
    return ms[min(len(ms) - 1, max(0, int(np.ceil(q * len(ms))) - 1))]


def batched_section(ctx, stream, steps: int, warmup: int, plain_steps: int) -> dict:
    """Batched workload: 512 aliased sets (sizes log-uniform in [1e3, 1e6],
    uniform / sphere / clumps), cluster size s = 64, built by one
    fmm_build_batched call per step, against the same sets built one
    fmm_build call at a time (per-instance plain launches)."""
    import torch
    from paper_1301_1704_gb300 import workloads
    sets, kinds = workloads.batch_sets(workloads.CONFIG_SEEDS[4])
    devs = [torch.from_numpy(p).cuda() for p in sets]
    pairs = [(d, d) for d in devs]
    npts = int(sum(len(p) for p in sets))  # aliased: each point counted once
    batch = ctx.batch(pairs)
    saved = ctx.tuning()
    tuned = ctx.autotune(batch, s=64, trials=2, stream=stream)

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        launches = 0
        torch.cuda.synchronize()
        for a, b in ev:
            a.record(stream)
            launches += fn()
            b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], launches

    def one_batched():
        ctx.build_batched(batch, s=64, stream=stream, raw=True)
        return ctx.last_launch_count()

    def one_plain():
        n = 0
        for d in devs:
            ctx.build(d, d, s=64, stream=stream, raw=True)
            n += ctx.last_launch_count()
        return n

    for _ in range(warmup):
        one_batched()
    bt, bl = timed(one_batched, steps)
    for _ in range(min(warmup, 2)):
        one_plain()
    pt, pl = timed(one_plain, plain_steps)
    out = {}
    for name, t, nl in (("batched", bt, bl), ("plain", pt, pl)):
        p50 = _pct(t, 0.5)
        out[name] = {"value": npts / (sum(t) / len(t) / 1e3) / 1e6, "unit": "Mpts/s",
                     "p50_ms": p50, "p99_ms": _pct(t, 0.99), "steps": len(t),
                     "gpu_launches_per_step": nl / len(t)}
    # Compulsory bytes of one batched build (aliased sets read and written once).
    outs = ctx.build_batched(batch, s=64, stream=stream, raw=True)
    torch.cuda.synchronize()
    alg, nnz2, nnz4, levels = 0, 0, 0, []
    for i in range(len(sets)):
        t = outs[i]
        n = t.n_src
        alg += 16 * n
        levels.append(t.L)
        for l in range(t.L + 1):
            alg += 16 * t.nbox_src[l] + 4
        for l in range(2, t.L + 1):
            nnz2 += t.nnz_e2[l]
            nnz4 += t.nnz_e4[l]
            alg += 8 * (t.nbox_recv[l] + 1)
    alg += 4 * (nnz2 + nnz4)
    peak, peak_kind = _peaks()
    ctx.reset_timing()
    ctx.set_timing(True)
    for _ in range(3):
        one_batched()
    torch.cuda.synchronize()
    ctx.set_timing(False)
    out["batched"]["kernel_ms_per_step"] = {k: v[1] / 3 for k, v in sorted(ctx.timing().items())}
    out["batched"]["build_roofline"] = {
        "alg_bytes": alg, "frac_of_peak": alg / (out["batched"]["p50_ms"] / 1e3) / 1e9 / peak,
        "peak": peak, "peak_kind": peak_kind, "note": "compulsory bytes / p50 step time"}
    out["nnz"] = {"e2": int(nnz2), "e4": int(nnz4)}
    out["levels"] = {"min": int(min(levels)), "max": int(max(levels)),
                     "mean": float(np.mean(levels))}
    out["batched"]["tuning"] = tuned
    ctx.set_tuning(saved["sort_kind"], saved["sort_items"])
    out["workload"] = ("512 aliased sets, sizes log-uniform in [1e3, 1e6], uniform / sphere / "
                       "clumps with p = 1/3, s = 64 (per-set L); batched = one fmm_build_batched "
                       "call, plain = one fmm_build call per set")
    out["points"] = npts
    out["speedup_vs_plain"] = out["batched"]["value"] / out["plain"]["value"]
    return out


SERVE_SIZES = (10_000, 10_000, 100_000, 100_000, 1_000_000, 1_000_000, 10_000_000, 10_000_000)
SERVE_RATE = 2000.0


def serve_trace(nsys: int, steps: int, rate: float, seed: int):
    """Poisson arrivals at `rate`/s, each for a uniformly chosen system,
    until every system has `steps` requests."""
    rng = np.random.default_rng(seed)
    per = np.zeros(nsys, np.int64)
    arr, sys_ = [], []
    t = 0.0
    while per.min() < steps:
        t += rng.exponential(1.0 / rate)
        k = int(rng.integers(0, nsys))
        arr.append(t)
        sys_.append(k)
        per[k] += 1
    return np.array(arr), np.array(sys_, np.uint32)


def _serve_run(fmmds, pts, levels, seed, arr, sys_, workers, batch) -> dict:
    srv = fmmds.Server(0, workers=workers, max_batch=batch)
    try:
        for k, (p, L) in enumerate(zip(pts, levels)):
            srv.add_system(p, L, 0.1, seed=seed * 1000 + k)
        infos = srv.run_trace(arr, sys_)
    finally:
        srv.close()
    lat = np.array([(i["t_done"] - i["t_arrival"]) * 1e3 for i in infos])
    span = max(i["t_done"] for i in infos) - min(i["t_arrival"] for i in infos)
    npts = sum(i["points"] for i in infos)
    return {"value": npts / span / 1e6, "unit": "Mpts/s",
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "requests": len(infos), "span_s": span,
            "mean_batch": float(np.mean([i["batch_size"] for i in infos])),
            "failed": int(sum(i["status"] != 0 for i in infos))}


def served_section(ctx, steps: int) -> dict:
    """Served dynamic rebuilds: 8 resident clump systems (two each of 1e4,
    1e5, 1e6, 1e7 points), depth fixed from the initial state at s = 64,
    Poisson requests, each advancing one random system by one step (Gaussian
    steps of 0.1 h_L, wall reflection) and rebuilding it.  Served =
    continuous batching over 2 concurrent workers; plain = one worker, one
    system per build (per-instance launches).  Two offered loads: the
    required 2000 requests/s (more points per second than the GPU builds, so
    queues grow over the trace and latency measures the backlog), and 60 % of
    the served throughput measured there (below capacity: latency is the
    service time)."""
    import torch
    from paper_1301_1704_gb300 import fmmds, workloads
    seed = workloads.CONFIG_SEEDS[5]
    pts = [workloads.clumps(n, seed * 1000 + k) for k, n in enumerate(SERVE_SIZES)]
    levels = []
    for p in pts:
        d = torch.from_numpy(p).cuda()
        levels.append(ctx.build(d, d, s=64).L)
        del d
    torch.cuda.synchronize()
    mean_pts = float(np.mean(SERVE_SIZES))
    out = {"offered_2000": {}, "below_capacity": {}}
    arr, sys_ = serve_trace(len(pts), steps, SERVE_RATE, seed)
    for name, workers, batch in (("served", 2, 8), ("plain", 1, 1)):
        out["offered_2000"][name] = _serve_run(fmmds, pts, levels, seed, arr, sys_, workers, batch)
    out["offered_2000"]["offered_mpts_s"] = SERVE_RATE * mean_pts / 1e6
    # below capacity: 60 % of the served throughput just measured
    rate = 0.6 * out["offered_2000"]["served"]["value"] * 1e6 / mean_pts
    low_steps = max(20, steps // 5)
    arr2, sys2 = serve_trace(len(pts), low_steps, rate, seed + 1)
    for name, workers, batch in (("served", 2, 8), ("plain", 1, 1)):
        out["below_capacity"][name] = _serve_run(fmmds, pts, levels, seed, arr2, sys2, workers,
                                                 batch)
    out["below_capacity"]["rate_per_s"] = rate
    out["below_capacity"]["offered_mpts_s"] = rate * mean_pts / 1e6
    out["below_capacity"]["steps_per_system"] = low_steps
    # Kernel breakdown of one batched build of all 8 systems (what a full
    # served batch runs, without the time step) and of the 1e7 system alone.
    devs = [torch.from_numpy(p).cuda() for p in pts]
    bd = {}
    for name, idx in (("batch_of_8", list(range(len(pts)))), ("one_1e7", [6])):
        b = ctx.batch([(devs[i], devs[i]) for i in idx], levels=[levels[i] for i in idx])
        for _ in range(3):
            ctx.build_batched(b, L=7, raw=True)
        torch.cuda.synchronize()
        ctx.reset_timing()
        ctx.set_timing(True)
        t0 = time.perf_counter()
        for _ in range(5):
            ctx.build_batched(b, L=7, raw=True)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / 5 * 1e3
        ctx.set_timing(False)
        kt = ctx.timing()
        npt = sum(len(pts[i]) for i in idx)
        bd[name] = {"points": npt, "wall_ms": wall, "value": npt / (wall / 1e3) / 1e6,
                    "kernel_ms": {k: v[1] / 5 for k, v in sorted(kt.items(), key=lambda kv: -kv[1][1])},
                    "kernel_sum_ms": sum(v[1] for v in kt.values()) / 5}
    out["batch_breakdown"] = bd
    del devs
    out["workload"] = ("8 resident clump systems (2 x 1e4, 1e5, 1e6, 1e7 points), L from the "
                       f"initial state at s = 64 ({levels}), Poisson requests each for a uniformly "
                       f"chosen system: {SERVE_RATE:.0f}/s until every system has {steps} steps, and "
                       f"{rate:.0f}/s until every system has {low_steps} steps; served = continuous "
                       "batching (2 workers, up to 8 systems per batched build), plain = 1 worker, "
                       "1 system per build")
    out["speedup_vs_plain"] = out["offered_2000"]["served"]["value"] / out["offered_2000"]["plain"]["value"]
    return out


def _timed(fn, steps: int, stream):
    """Per-step CUDA-event times (ms) of `steps` calls of fn on `stream`, the
    whole region's time, and the kernel launches fn reports."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    torch.cuda.synchronize()
    t0.record(stream)
    for a, b in ev:
        a.record(stream)
        launches += fn()
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], t0.elapsed_time(t1), launches


def small_config_section(ctx, stream, steps: int) -> dict:
    """Config 1: N = M = 16384 uniform, L = 4 (a few MB: launch-latency
    bound, so microseconds per build, eagerly and in graph mode; a roofline
    fraction would mean nothing here)."""
    import torch
    from paper_1301_1704_gb300 import workloads
    src_h, recv_h, L = workloads.config_inputs(1)
    src, recv = torch.from_numpy(src_h).cuda(), torch.from_numpy(recv_h).cuda()
    out = {"workload": "config 1: N=M=16384 uniform [0,1)^3 float32, L=4, lists at levels 2..4"}
    for mode in ("eager", "graph"):
        ctx.set_graphs(mode == "graph")

        def one():
            ctx.build(src, recv, L=L, stream=stream, raw=True)
            return ctx.last_launch_count()

        for _ in range(5):
            one()
        t, _, nl = _timed(one, steps, stream)
        out[mode] = {"p50_us": 1e3 * _pct(t, 0.5), "p99_us": 1e3 * _pct(t, 0.99),
                     "value": 2 * len(src_h) / (_pct(t, 0.5) / 1e3) / 1e6, "unit": "Mpts/s",
                     "steps": steps, "gpu_launches_per_step": nl / steps}
    ctx.set_graphs(False)
    out["graph_stats"] = ctx.graph_stats()
    return out


def sparse_config_section(ctx, stream, steps: int, warmup: int, autotune: bool) -> dict:
    """Config 3: N = M = 2^24, half on a sphere surface, half in 64 clumps,
    L = 9 (most boxes empty): Mpoints/s, p50/p99, and the whole build's
    fraction of the HBM roofline on its compulsory bytes."""
    import torch
    from paper_1301_1704_gb300 import workloads
    src_h, recv_h, L = workloads.config_inputs(3)
    src, recv = torch.from_numpy(src_h).cuda(), torch.from_numpy(recv_h).cuda()
    saved = ctx.tuning()
    tuned = ctx.autotune([(src, recv)], L=L, trials=2, stream=stream) if autotune else None

    def one():
        ctx.build(src, recv, L=L, stream=stream, raw=True)
        return ctx.last_launch_count()

    for _ in range(warmup):
        one()
    t, total, nl = _timed(one, steps, stream)
    tree = ctx.build(src, recv, L=L, stream=stream)
    torch.cuda.synchronize()
    alg = _algorithmic_bytes(tree)
    peak, peak_kind = _peaks()
    ms = total / steps
    ctx.set_tuning(saved["sort_kind"], saved["sort_items"])
    return {"workload": "config 3: N=M=2^24, half on a sphere surface (r=0.4, jitter 1e-3), "
                        "half in 64 Gaussian clumps (sigma 0.01), L=9, lists at levels 2..9",
            "value": 2 * len(src_h) / (ms / 1e3) / 1e6, "unit": "Mpts/s", "ms_per_step": ms,
            "p50_ms": _pct(t, 0.5), "p99_ms": _pct(t, 0.99), "steps": steps,
            "gpu_launches_per_step": nl / steps, "tuning": tuned,
            "roofline": {"bound": "hbm", "alg_bytes": alg["total"],
                         "achieved": alg["total"] / (ms / 1e3) / 1e9, "peak": peak,
                         "frac": alg["total"] / (ms / 1e3) / 1e9 / peak,
                         "peak_kind": peak_kind, "unit": "GB/s"},
            "boxes": {"finest_src": int(tree.src.nbox[L]), "finest_recv": int(tree.recv.nbox[L])},
            "nnz": {"e2": int(sum(tree.nnz_e2)), "e4": int(sum(tree.nnz_e4))}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--points", type=int, default=N_PTS,
                    help="points per set (default 2^24; smaller values only for profiling)")
    ap.add_argument("--level", type=int, default=LEVEL)
    ap.add_argument("--sort-kind", type=int, default=None,
                    help="sort kind (see fmm_set_tuning; else autotuned)")
    ap.add_argument("--sort-items", type=int, default=0, help="points per thread of a sort tile")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tuning")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison of the sort kinds")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-graphs", action="store_true", help="skip the graph-mode timings")
    ap.add_argument("--no-configs", action="store_true", help="skip the config 1 and 3 timings")
    ap.add_argument("--clock-window", type=float, default=1.0,
                    help="seconds of untimed builds, under the clock sampler, before the timed "
                         "region")
    ap.add_argument("--plain-steps", type=int, default=5,
                    help="steps of the per-instance comparison of the batched workload")
    ap.add_argument("--serve-steps", type=int, default=1000,
                    help="time steps per system of the served workload (0: skip it)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.warmup < 3:
        raise SystemExit("warmup must be >= 3")

    import torch
    from paper_1301_1704_gb300 import fmmds, workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    npts, level = args.points, args.level
    full = (npts, level) == (N_PTS, LEVEL)
    src_h = workloads.uniform(npts, SEEDS[0])
    recv_h = workloads.uniform(npts, SEEDS[1])
    src = torch.from_numpy(src_h).cuda()
    recv = torch.from_numpy(recv_h).cuda()
    ctx = fmmds.Context(local)
    stream = torch.cuda.current_stream()
    autotuned = None
    if args.sort_kind is not None:
        ctx.set_tuning(args.sort_kind, args.sort_items)
    elif not args.no_autotune:
        # the library's autotuner picks the sort kind and tile size on these inputs
        autotuned = ctx.autotune([(src, recv)], L=level, trials=3, stream=stream)

    def one():
        ctx.build(src, recv, L=level, stream=stream, raw=True)
        return ctx.last_launch_count()

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()

    # Clock record: the sampler runs over `--clock-window` seconds of untimed
    # builds right before the timed region and over the timed region itself
    # (a timed region of a few dozen builds lasts only a few sampling periods).
    clocks = ClockSampler(local)
    clocks.start()
    t_end = time.time() + args.clock_window
    while time.time() < t_end:
        for _ in range(20):
            one()
        torch.cuda.synchronize()
    # Timed region: K builds through the C ABI (raw result struct: no Python
    # wrapping of the outputs), CUDA events on the build's stream.
    barrier()
    step_ms, total_ms, launches = _timed(one, args.steps, stream)
    barrier()
    clk = clocks.stop()
    clk["window"] = f"{args.clock_window:.1f} s of back-to-back builds, then the timed region"
    step_ms = sorted(step_ms)

    # Kernel durations: the same K builds again with the library's per-launch
    # events on (they add a little time, so they are kept out of `value`).
    ctx.reset_timing()
    ctx.set_timing(True)
    for _ in range(args.steps):
        one()
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ktimes = ctx.timing()

    # Graph mode (fmm_set_graphs): the same builds with their stream work
    # recorded into CUDA graphs that are updated and launched every build.
    graphs = None
    if not args.no_graphs:
        ctx.set_graphs(True)
        for _ in range(max(3, args.warmup)):
            one()
        g_ms, g_total, _ = _timed(one, args.steps, stream)
        graphs = {"p50_ms": _pct(g_ms, 0.5), "p99_ms": _pct(g_ms, 0.99),
                  "value": 2 * npts * args.steps / (g_total / 1e3) / 1e6, "unit": "Mpts/s",
                  "steps": args.steps, "graph_stats": ctx.graph_stats()}
        ctx.set_graphs(False)
    tree = ctx.build(src, recv, L=level, stream=stream)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, dist)

    pts_per_step = npts * 2
    value = replica_throughput(pts_per_step * args.steps, total_ms, ws) / 1e6
    ms_per_step = total_ms / args.steps

    # Roofline of the whole build (the unit one step processes): compulsory
    # bytes -- inputs read once, outputs written once -- over the measured
    # time per build, against the measured copy bandwidth.
    peak, peak_kind = _peaks()
    alg = _algorithmic_bytes(tree)
    achieved = alg["total"] / (ms_per_step / 1e3) / 1e9
    wl_key = "plain_uniform_2p24_L7" if full else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": _build_traffic(wl_key) if wl_key else None,
                "kernel": "whole build (every kernel of one fmm_build)", "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg["total"], "alg_bytes": alg,
                "avg_launch_ms": ms_per_step,
                "frac_of_nominal_8000": achieved / 8000.0}
    per_kernel = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps,
                      "share": v[1] / sum(x[1] for x in ktimes.values())}
                  for k, v in sorted(ktimes.items(), key=lambda kv: -kv[1][1])}

    # End to end through the C ABI: pinned host inputs, copies inside the call.
    hs = torch.from_numpy(src_h).pin_memory()
    hr = torch.from_numpy(recv_h).pin_memory()

    def one_e2e():
        ctx.build(hs, hr, L=level, flags=fmmds.FMM_FLAG_HOST_INPUT, stream=stream, raw=True)
        return 0

    for _ in range(min(2, args.e2e_steps)):
        one_e2e()
    barrier()
    e2e_val = None
    if args.e2e_steps:
        _, e2e_ms, _ = _timed(one_e2e, args.e2e_steps, stream)
        e2e_ms = max_over_ranks(max(e2e_ms, 1e-9), dist)
        e2e_val = replica_throughput(pts_per_step * args.e2e_steps, e2e_ms, ws) / 1e6
    # The same build with each way of ordering the points.
    sort_kinds = {}
    if full and not args.no_compare:
        base = ctx.tuning()
        for kind, name in ((fmmds.FMM_SORT_RTS, "radix_rts"),
                           (fmmds.FMM_SORT_ONESWEEP, "radix_onesweep"),
                           (fmmds.FMM_SORT_FIXED_GRID, "fixed_grid")):
            ctx.set_tuning(kind)
            for _ in range(2):
                one()
            t, _, _ = _timed(one, 5, stream)
            sort_kinds[name] = _pct(t, 0.5)
        ctx.set_tuning(base["sort_kind"], base["sort_items"])
    configs = {}
    if not args.no_configs and rank == 0:
        configs["config1"] = small_config_section(ctx, stream, max(args.steps, 200))
        configs["config3"] = sparse_config_section(ctx, stream, args.steps, args.warmup,
                                                   not args.no_autotune)
    nnz = {"e2": int(sum(tree.nnz_e2)), "e4": int(sum(tree.nnz_e4))}
    tuning_now = ctx.tuning()
    batched = None
    if not args.no_batched:
        batched = batched_section(ctx, stream, args.steps, args.warmup, args.plain_steps)
    served = None
    if args.serve_steps > 0 and rank == 0:
        # the served workload gets the device to itself: this context's arena
        # and PyTorch's cached blocks are released first
        del tree
        ctx.close()
        torch.cuda.empty_cache()
        sctx = fmmds.Context(local)
        served = served_section(sctx, args.serve_steps)
        sctx.close()
        ctx = None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "tuning": dict(tuning_now, autotuned=autotuned is not None),
            "config": {"workload": WORKLOAD if full else
                       f"profiling case N=M={npts} uniform, L={level}", "N": npts, "M": npts, "L": level,
                       "seeds": list(SEEDS), "l2": "inputs larger than L2 (402 MB of xyz)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "p50_ms": _pct(step_ms, 0.5), "p99_ms": _pct(step_ms, 0.99),
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": roofline,
            "kernels": per_kernel,
            "nnz": nnz,
            "e2e": {"value": e2e_val, "unit": "Mpts/s", "h2d_bytes_per_step": 12 * pts_per_step,
                    "d2h_bytes_per_step": D2H_BYTES, "steps": args.e2e_steps},
        }
        if not args.no_cpu_baseline and ws == 1 and full:
            line["cpu_baseline"] = cpu_baseline()
        if sort_kinds:
            line["p50_ms_by_sort_kind"] = sort_kinds
        if graphs is not None:
            line["graph_mode"] = graphs
        line.update(configs)
        if batched is not None:
            line["batched"] = batched
        if served is not None:
            line["served"] = served
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
