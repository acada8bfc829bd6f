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

    INTERVAL_MS = 100

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


def _kernel_alg_bytes(name: str, tree) -> float | None:
    """Algorithmic bytes of ALL launches of one kernel in one build (None if
    the kernel has no compulsory traffic of its own)."""
    n, m = tree.src.n, tree.recv.n
    if name == "list_fill":  # writes the E2 and E4 index lists (offsets come from the scans)
        return 4 * sum(tree.nnz_e2[l] + tree.nnz_e4[l] for l in range(2, tree.L + 1))
    if name in ("onesweep", "rts_scatter"):  # one LSD pass reads and writes (u64 key, u32 index)
        return None  # filled in by the caller from the pass count
    if name == "tile_hist":  # reads the keys (or the coordinates in the first pass)
        return None
    if name == "finish_boxes":  # reads (key, index), writes the permutation and every box level
        bx = 0
        for sd in (tree.src, tree.recv):
            for l in range(tree.L + 1):
                nb = sd.nbox[l]
                bx += 8 * nb + 4 * (nb + 1) + 4 * nb + (4 * (nb + 1) if l < tree.L else 0)
        return 16 * (n + m) + bx
    if name == "upfront_hist":  # reads the coordinates
        return 12 * (n + m)
    return None


def _src_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1301_1704_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic_for(kernel: str):
    """ncu DRAM bytes per launch of `kernel`, if captured from the current source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    e = d.get(kernel)
    if not e or e.get("src_hash") != _src_hash():
        return None
    return e.get("dram_bytes_per_launch")


def cpu_baseline(sub: int = 1) -> dict:
    """The oracle on the points of the workload that fall in the sub-cube
    [0, 1/sub)^3 (same level, same density, 1/sub^3 of the work; the whole
    workload by default, about 25 s on one core): its OpenMP build on all
    host cores, and the plain build on one core."""
    from oracle import oracle
    from paper_1301_1704_gb300 import workloads
    src = workloads.uniform(N_PTS, SEEDS[0])
    recv = workloads.uniform(N_PTS, SEEDS[1])
    lim = np.float32(1.0 / sub)
    s = np.ascontiguousarray(src[np.all(src < lim, axis=1)])
    r = np.ascontiguousarray(recv[np.all(recv < lim, axis=1)])
    pts = len(s) + len(r)
    out = {}
    for parallel in (True, False):
        oracle.build(parallel=parallel)
        t0 = time.perf_counter()
        oracle.build_tree(s, r, L=LEVEL, mode=oracle.MODE_STENCIL, parallel=parallel)
        out[parallel] = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    return {"value": pts / out[True] / 1e6, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
            "sample": f"points of the benchmark inputs inside [0,1/{sub})^3 ({len(s)} src + {len(r)} recv),"
                      f" L={LEVEL}, stencil lists; the oracle's OpenMP build on {cores} threads:"
                      f" {out[True]:.1f} s",
            "single_thread": {"value": pts / out[False] / 1e6, "cores": 1,
                              "seconds": out[False]}}


def reference_arm(args) -> None:
    """`--impl reference`: the CPU oracle (its OpenMP build, all host cores),
    each step one bounded sample of the workload (points inside one of the 64
    sub-cubes of side 1/4, in turn)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import oracle
    from paper_1301_1704_gb300 import workloads
    oracle.build(parallel=True)
    cores = os.cpu_count() or 1
    src = workloads.uniform(N_PTS, SEEDS[0])
    recv = workloads.uniform(N_PTS, SEEDS[1])
    cs, cr = (src * 4).astype(np.int64).clip(0, 3), (recv * 4).astype(np.int64).clip(0, 3)
    ids = cs[:, 0] + 4 * cs[:, 1] + 16 * cs[:, 2]
    idr = cr[:, 0] + 4 * cr[:, 1] + 16 * cr[:, 2]
    times, pts = [], []
    for step in range(args.warmup + args.steps):
        sub = step % 64
        s = np.ascontiguousarray(src[ids == sub])
        r = np.ascontiguousarray(recv[idr == sub])
        t0 = time.perf_counter()
        oracle.build_tree(s, r, L=LEVEL, mode=oracle.MODE_STENCIL, parallel=True)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            pts.append(len(s) + len(r))
    total = sum(times)
    val = sum(pts) / total / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "one 1/64 sub-cube of the inputs per step"},
        "cpu_baseline": {"value": val, "unit": "Mpts/s", "cores": cores, "kind": "oracle",
                         "sample": "per step: the points of the benchmark inputs inside one of the"
                                   " 64 sub-cubes of side 1/4 (about 2^18 per set), L=7; the"
                                   f" oracle's OpenMP build on {cores} threads"},
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


def served_section(ctx, steps: int) -> dict:
    """Served dynamic rebuilds: 8 resident clump systems (two each of 1e4,
    1e5, 1e6, 1e7 points), depth fixed from the initial state at s = 64,
    Poisson requests at 2000/s, each advancing one random system by one step
    (Gaussian steps of 0.1 h_L, wall reflection) and rebuilding it.  Served =
    continuous batching over 2 concurrent workers; plain = one worker, one
    system per build (per-instance launches)."""
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
    arr, sys_ = serve_trace(len(pts), steps, SERVE_RATE, seed)
    out = {}
    for name, workers, batch in (("served", 2, 8), ("plain", 1, 1)):
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
        out[name] = {"value": npts / span / 1e6, "unit": "Mpts/s",
                     "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)),
                     "requests": len(infos), "span_s": span,
                     "mean_batch": float(np.mean([i["batch_size"] for i in infos])),
                     "failed": int(sum(i["status"] != 0 for i in infos))}
    out["workload"] = ("8 resident clump systems (2 x 1e4, 1e5, 1e6, 1e7 points), L from the "
                       f"initial state at s = 64 ({levels}), Poisson {SERVE_RATE:.0f}/s requests "
                       f"until every system has {steps} steps; served = continuous batching "
                       "(2 workers, up to 8 systems per batched build), plain = 1 worker, "
                       "1 system per build")
    out["speedup_vs_plain"] = out["served"]["value"] / out["plain"]["value"]
    return out


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
                    help="0 radix reduce-then-scan, 1 radix onesweep, 2 Fixed-Grid (else autotuned)")
    ap.add_argument("--sort-items", type=int, default=0, help="points per thread of a sort tile")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tuning")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison of the sort kinds")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-graphs", action="store_true", help="skip the graph-mode timings")
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

    for _ in range(args.warmup):
        ctx.build(src, recv, L=level, stream=stream, raw=True)
    torch.cuda.synchronize()

    # Timed region: K builds through the C ABI (raw result struct: no Python
    # wrapping of the outputs), CUDA events on the build's stream.
    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    barrier()
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for i in range(args.steps):
        starts[i].record(stream)
        ctx.build(src, recv, L=level, stream=stream, raw=True)
        ends[i].record(stream)
        launches += ctx.last_launch_count()
    t_all1.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = t_all0.elapsed_time(t_all1)
    step_ms = sorted(s.elapsed_time(e) for s, e in zip(starts, ends))

    # Kernel durations: the same K builds again with the library's per-launch
    # events on (they add a little time, so they are kept out of `value`).
    ctx.reset_timing()
    ctx.set_timing(True)
    for i in range(args.steps):
        ctx.build(src, recv, L=level, stream=stream, raw=True)
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ktimes = ctx.timing()

    # Graph mode (fmm_set_graphs): the same builds with their stream work
    # recorded into CUDA graphs that are updated and launched every build.
    graphs = None
    if not args.no_graphs:
        ctx.set_graphs(True)
        for _ in range(max(3, args.warmup)):
            ctx.build(src, recv, L=level, stream=stream, raw=True)
        torch.cuda.synchronize()
        for i in range(args.steps):
            starts[i].record(stream)
            ctx.build(src, recv, L=level, stream=stream, raw=True)
            ends[i].record(stream)
        torch.cuda.synchronize()
        g_ms = sorted(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends))
        graphs = {"p50_ms": g_ms[len(g_ms) // 2], "p99_ms": g_ms[-1],
                  "value": 2 * npts / (g_ms[len(g_ms) // 2] / 1e3) / 1e6, "unit": "Mpts/s",
                  "steps": args.steps, "graph_stats": ctx.graph_stats()}
        ctx.set_graphs(False)
    tree = ctx.build(src, recv, L=level, stream=stream)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, dist)

    pts_per_step = npts * 2
    value = replica_throughput(pts_per_step * args.steps, total_ms, ws) / 1e6
    p50 = step_ms[len(step_ms) // 2]
    p99 = step_ms[min(len(step_ms) - 1, int(np.ceil(0.99 * len(step_ms))) - 1)]

    # Roofline of the dominant kernel (largest summed time in the timed region).
    peak, peak_kind = _peaks()
    alg = _algorithmic_bytes(tree)
    def alg_of(name):
        # A radix pass reads and writes (u64 key, u32 index) per point;
        # rts_scatter sorts both sets in one launch per pass, onesweep one set
        # per launch (and forms the keys from the coordinates in its pass 0).
        per_build = ktimes[name][0] / args.steps
        if name == "rts_scatter":  # pass 0 reads the stored 8-byte keys: 20 bytes a point
            return pts_per_step * (20 + 24 * (per_build - 1))
        if name == "onesweep":
            return 24 * pts_per_step * per_build / 2
        if name == "tile_hist":  # first pass reads the coordinates, later ones the keys
            return pts_per_step * (12 + 8 * (per_build - 1))
        return _kernel_alg_bytes(name, tree)

    measured = {k: v for k, v in ktimes.items() if alg_of(k) is not None}
    dom_name, (dom_launches, dom_ms) = max(measured.items(), key=lambda kv: kv[1][1])
    per_build_launches = dom_launches / args.steps
    avg_ms = dom_ms / dom_launches
    bytes_per_launch = alg_of(dom_name) / per_build_launches
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": _traffic_for(dom_name),
                "kernel": dom_name, "peak_kind": peak_kind,
                "alg_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms}
    kernel_frac = {k: alg_of(k) / (v[1] / args.steps / 1e3) / 1e9 / peak
                   for k, v in measured.items()}
    build_frac = alg["total"] / (p50 / 1e3) / 1e9 / peak

    # End to end through the C ABI: pinned host inputs, copies inside the call.
    hs = torch.from_numpy(src_h).pin_memory()
    hr = torch.from_numpy(recv_h).pin_memory()
    for _ in range(min(2, args.e2e_steps)):
        ctx.build(hs, hr, L=level, flags=fmmds.FMM_FLAG_HOST_INPUT, stream=stream, raw=True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        ctx.build(hs, hr, L=level, flags=fmmds.FMM_FLAG_HOST_INPUT, stream=stream, raw=True)
    e1.record(stream)
    barrier()
    e2e_ms = max(e0.elapsed_time(e1), 1e-9)
    e2e_ms = max_over_ranks(e2e_ms, dist)
    e2e_val = (replica_throughput(pts_per_step * args.e2e_steps, e2e_ms, ws) / 1e6
               if args.e2e_steps else None)
    # The same build with each way of ordering the points (radix passes in
    # reduce-then-scan or onesweep form, the paper's Fixed-Grid pseudo-sort).
    sort_kinds = {}
    if (npts, level) == (N_PTS, LEVEL) and not args.no_compare:
        base = ctx.tuning()
        for kind, name in ((fmmds.FMM_SORT_RTS, "radix_rts"), (fmmds.FMM_SORT_ONESWEEP, "radix_onesweep"),
                           (fmmds.FMM_SORT_FIXED_GRID, "fixed_grid")):
            ctx.set_tuning(kind)
            for _ in range(2):
                ctx.build(src, recv, L=level, stream=stream, raw=True)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(5)]
            for a, b in evs:
                a.record(stream)
                ctx.build(src, recv, L=level, stream=stream, raw=True)
                b.record(stream)
            torch.cuda.synchronize()
            sort_kinds[name] = _pct([a.elapsed_time(b) for a, b in evs], 0.5)
        ctx.set_tuning(base["sort_kind"], base["sort_items"])
    batched = None
    if not args.no_batched:
        batched = batched_section(ctx, stream, args.steps, args.warmup, args.plain_steps)
    served = None
    if args.serve_steps > 0 and rank == 0:
        served = served_section(ctx, args.serve_steps)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpts/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "tuning": dict(ctx.tuning(), autotuned=autotuned is not None),
            "config": {"workload": WORKLOAD if (npts, level) == (N_PTS, LEVEL) else
                       f"profiling case N=M={npts} uniform, L={level}", "N": npts, "M": npts, "L": level,
                       "seeds": list(SEEDS), "l2": "inputs larger than L2 (402 MB of xyz)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "p50_ms": p50, "p99_ms": p99,
            "gpu_launches": launches,
            "clocks": clk,
            "roofline": roofline,
            "build_roofline": {"alg_bytes": alg, "frac_of_peak": build_frac, "peak": peak,
                               "note": "whole build, compulsory bytes / p50 step time"},
            "kernel_ms_per_step": {k: v[1] / args.steps for k, v in sorted(ktimes.items())},
            "kernel_hbm_frac": kernel_frac,
            "nnz": {"e2": int(sum(tree.nnz_e2)), "e4": int(sum(tree.nnz_e4))},
            "e2e": {"value": e2e_val, "unit": "Mpts/s", "h2d_bytes_per_step": 12 * pts_per_step,
                    "d2h_bytes_per_step": D2H_BYTES, "steps": args.e2e_steps},
        }
        if not args.no_cpu_baseline and ws == 1 and (npts, level) == (N_PTS, LEVEL):
            line["cpu_baseline"] = cpu_baseline()
        if sort_kinds:
            line["p50_ms_by_sort_kind"] = sort_kinds
        if graphs is not None:
            line["graph_mode"] = graphs
        if batched is not None:
            line["batched"] = batched
        if served is not None:
            line["served"] = served
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
