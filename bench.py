"""Benchmark: Monte Carlo Heston price + Greeks on GB300.

One step = one full estimate of the multi-strike workload: 2^22 paths x 252
steps, European + arithmetic Asian (252 equal dates) calls at K in
{90, 100, 110} (36 estimates with standard errors), FP32 path recursion with
FP64 sums, Philox normals, full truncation.  The step is the path kernel
(heston_mc_launch_tiles) plus the fixed-order reduction
(heston_mc_reduce_tiles), i.e. what heston_mc_launch enqueues.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  `value` is path-steps/s over all ranks with inputs
resident on the device; `e2e` is the same metric through the synchronous
host API (heston_mc_price_greeks_ex: host structs in, results copied back).
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "path-steps/s at fixed std error (Greek-sets/s alongside)"
UNIT = "path-steps/s"

# Algorithmic work per path-step for this workload (FP32 path, full
# truncation, European + Asian with a date every step, Vega/Theta tangents,
# Gamma weights).  The roofline's per-unit figure is the method's count, one
# issue slot per operation: Philox4x32-10 half a block ~45 INT32 operations
# (10 rounds x 2 wide multiplies + ~6 xors/adds, per 2 steps), Box-Muller 4
# MUFU + ~6 FP32, correlation and W 3, log-price 1 MUFU + ~4, variance ~7,
# Asian date 1 MUFU + 3, Vega/Theta tangents ~16, Gamma weight 2: about 45
# INT32 + 41 FP32 + 6 MUFU = 92 slots per path-step (88 without an Asian
# date).
METHOD_SLOTS_PER_PATH_STEP = 92
METHOD_SLOTS_NO_DATE = 88
# The path kernel's own formulation needs fewer:
#   82.25 scalar operations.  38.25 cannot pack: Philox4x32-10 16 (per path
#   and block of 2 steps, 15 wide multiplies and 17 xors: the path's R1
#   product is loop-invariant and the products of the warp-uniform (step
#   pair, high path word) come from a per-warp table), the table's 128-bit
#   load per lane and step pair 0.25, uniform masks + conversions 4,
#   Box-Muller lg2/sqrt/sin/cos 4 + compare and two factor selects 3,
#   truncation compare/max/selects 6 (the mean-reversion factor's included)
#   + rsqrt 1, Milstein-term selects 2, Asian ex2 1, loop 1.  44 are FP32
#   adds / multiplies / FMAs (uniform scaling 2, Box-Muller 8, step 29, Asian
#   date 5), which sm_100's f32x2 instructions retire two per issue slot.
# Its issue-slot minimum is therefore 38.25 + 44/2 = 60.25 thread-instruction
# slots per path-step against 1 slot per lane per clock.
ALGO_OPS_PER_PATH_STEP = 82.25
ALGO_SLOTS_PER_PATH_STEP = 60.25
# The persistent batched kernel runs Philox without the table: 20 per
# path-step (10 wide multiplies and 10 xors), 64 slots with an Asian date
# every step and 3.5 fewer (ex2 + 5 FP32) without one.
BATCH_SLOTS_PER_PATH_STEP = 64.0
ISSUE_LANES_PER_SM_CLK = 128          # 4 SM sub-partitions x 1 warp-instruction x 32 lanes
# FP64 path (one European call): the explicit FP64 arithmetic per path-step,
# counted from the operations the method needs -- the Milstein step with its
# tangents and Gamma weights 38 (the correlation 4, V+ dt and u 2, du/dv0 and
# du/dT 6, Gamma weights 2, ln S and its tangents 8, V and its tangents 13,
# the Milstein term 3) and Box-Muller 9 (two int->double conversions, five
# scalings and products, two final products) -- 47, plus five FP64 special
# functions (log, sqrt, sin and cos of 2 pi u2, 1 / sqrt(V dt)) that run on
# the same pipe and are not counted.
FP64_OPS_PER_PATH_STEP = 47
# The FMA pipe's heavy half, which binds the FP32 path kernel: per warp and
# lane-step (32 lanes x 2 paths = 64 path-steps) the lane's 15 Philox wide
# multiplies take about 4 of its cycles each and its 44 f32x2 FMA-pipe
# instructions 2 each (pipe micro-benchmarks): 148 cycles, one heavy half per
# SM sub-partition.
HEAVY_CYCLES_PER_LANE_STEP = 148
HEAVY_LANE_STEP_PATHS = 64
# The same mix measured: the heavy_mix micro-benchmark runs one lane's FMA-pipe
# work per step (15 wide multiplies + 44 f32x2 FMAs = 59 instructions, two
# path-steps) on independent chains; its rate / 59 x 2 is the path-steps/s
# ceiling of that mix on this GPU.
MIX_INSTS_PER_UNIT = 59
MIX_PATH_STEPS_PER_UNIT = 2
FLUSH_BYTES = 256 << 20               # > 129 MB L2
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "heston_paths_kernel_multi_strike_2p22.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2309_10477_gb300", "csrc", f)
                  for f in ("heston_device.cuh", "philox.cuh", "bm64_tables.h")]


def _dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.rows = []
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, on: bool):
        self.marks.append((time.time(), on))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary_between(self, t0, t1):
        """Median SM clock of the samples taken between host times t0 and t1."""
        sm = []
        for t, r in self.rows:
            if t0 <= t <= t1:
                try:
                    sm.append(float(r[1]))
                except (ValueError, IndexError):
                    pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "samples": len(sm)}

    def summary(self):
        windows = []
        for (t0, a), (t1, b) in zip(self.marks[::2], self.marks[1::2]):
            windows.append((t0, t1))
        inside = [r for t, r in self.rows if any(a <= t <= b for a, b in windows)]
        rows = inside or [r for _, r in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def _source_hash():
    """sha256[:16] of the device sources (heston_device.cuh, philox.cuh,
    bm64_tables.h, concatenated in that order): a committed ncu summary's
    figures are used only while it names the current hash."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


FP64_PROFILE = os.path.join(ROOT, "profiles", "heston_paths_kernel_fp64_single_european_2p16.md")


def _profile_value(path, pattern):
    """A number from a committed ncu summary, or None if the device source
    changed since it was captured."""
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"source sha256\[:16\]:\s*([0-9a-f]{16})", text)
    v = re.search(pattern, text)
    if not m or not v or m.group(1) != _source_hash():
        return None
    return float(v.group(1))


def _profiled_traffic():
    """DRAM bytes per launch of the path kernel from the committed ncu summary,
    or None if the kernel source changed since it was captured."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"source sha256\[:16\]:\s*([0-9a-f]{16})", text)
    t = re.search(r"dram bytes per full launch:\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != _source_hash():
        return None
    return float(t.group(1))


# ---------------------------------------------------------------------------
# Oracle (CPU) timing -- the reported baseline and the reference arm
# ---------------------------------------------------------------------------

def _oracle_sample(target_s: float):
    import oracle
    from paper_2309_10477_gb300 import workloads as wl
    w = wl.multi_strike_fp32()
    P = oracle.Params(**w.params)
    cs = [oracle.Contract(c[0], c[1], c[2], c[3], c[4]) for c in w.contracts]
    threads = oracle.max_threads()
    n = 4096 * threads
    oracle.mc_sums(P, cs, n, w.n_steps, w.seed)          # warm the threads
    t0 = time.perf_counter()
    oracle.mc_sums(P, cs, n, w.n_steps, w.seed)
    dt = time.perf_counter() - t0
    n_sample = int(min(n * target_s / max(dt, 1e-6), w.n_paths))
    n_sample = max(4096, (n_sample // 4096) * 4096)
    return w, P, cs, threads, n_sample


def _time_oracle(w, P, cs, n_sample, reps=1):
    import oracle
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.mc_sums(P, cs, n_sample, w.n_steps, w.seed)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return n_sample * w.n_steps / best, best


def host_info():
    """nproc, the CPU model and its maximum clock, from os and lscpu."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            k, v = k.strip(), v.strip()
            if k == "Model name":
                info["model"] = v
            elif k == "CPU max MHz":
                info["max_mhz"] = float(v)
            elif k == "Architecture":
                info["arch"] = v
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    return info


def _timed(fn):
    t0 = time.perf_counter()
    fn()
    return time.perf_counter() - t0


def cpu_baselines(budget_s: float = 3.0):
    """The oracle, as it stands, beside each configuration, on all host cores
    and on one: path-steps/s and Greek-sets/s (the oracle's SE at the same
    path count is the SE target, so these are rates at the same SE).  Each
    sample is sized to about budget_s seconds."""
    import oracle
    from paper_2309_10477_gb300 import workloads as wl
    all_threads = oracle.max_threads()
    out = {"host": host_info(), "threads_all": all_threads}

    def rate(run, n_full, path_steps_per_path, label, greek_sets):
        res = {}
        for mode, threads in (("all_cores", all_threads), ("one_core", 1)):
            oracle.set_threads(threads)
            try:
                n = 4096 * threads
                dt = _timed(lambda: run(n))
                n = int(min(n_full, max(4096, n * budget_s / max(dt, 1e-6))) // 4096 * 4096) or 4096
                dt = _timed(lambda: run(n))
            finally:
                oracle.set_threads(0)
            ps = n * path_steps_per_path / dt
            res[mode] = {"path_steps_per_s": ps, "cores": threads,
                         "greek_sets_per_s": greek_sets * ps / (n_full * path_steps_per_path),
                         "sample": f"{n} of {n_full} paths ({dt:.1f} s)"}
        res["workload"] = label
        return res

    # config 1: one European call, 2^16 x 100, FP64
    w1 = wl.single_european_fp64()
    P1, C1 = oracle.Params(**w1.params), [oracle.Contract(*c) for c in w1.contracts]
    out["single_european_fp64"] = rate(lambda n: oracle.mc_sums(P1, C1, n, w1.n_steps, w1.seed),
                                       w1.n_paths, w1.n_steps, w1.name, 1)
    # config 2: the headline workload
    w2 = wl.multi_strike_fp32()
    P2, C2 = oracle.Params(**w2.params), [oracle.Contract(*c) for c in w2.contracts]
    out["multi_strike"] = rate(lambda n: oracle.mc_sums(P2, C2, n, w2.n_steps, w2.seed),
                               w2.n_paths, w2.n_steps, w2.name, len(C2))
    # config 3: a 64-contract subset of the batched mix (every 16th contract), each
    # contract's paths capped to the sample, scaled by path-steps to the whole mix
    mix = wl.batched_contracts(1024)
    sub = mix[::16]
    total_ps = sum(d["n_paths"] * d["n_steps"] for d in mix)

    def run_mix(cap):
        for d in sub:
            oracle.mc_sums(oracle.Params(**d["params"]), [oracle.Contract(*d["contract"])],
                           min(cap, d["n_paths"]), d["n_steps"], 42)
    res3 = {}
    for mode, threads in (("all_cores", all_threads), ("one_core", 1)):
        # each contract's paths are capped at one 4096-path chunk per thread, so that
        # every thread has work on the contracts large enough to need it
        cap = 4096 * threads
        oracle.set_threads(threads)
        try:
            dt = _timed(lambda: run_mix(cap))
        finally:
            oracle.set_threads(0)
        ps = sum(min(cap, d["n_paths"]) * d["n_steps"] for d in sub) / dt
        res3[mode] = {"path_steps_per_s": ps, "cores": threads,
                      "greek_sets_per_s": 1024 * ps / total_ps,
                      "sample": f"64 of the 1024 contracts (every 16th), up to {cap} paths each "
                                f"({dt:.1f} s), scaled by path-steps to the whole mix"}
    res3["workload"] = "1024-contract batched mix (64-contract subset)"
    out["batched_mix"] = res3
    # config 4: the gradient (7 tangent directions) of the 252-step Asian call, 2^20 paths
    c4 = oracle.Contract(1, 100.0, 1.0)
    out["adjoint_gradient"] = rate(lambda n: oracle.mc_gradient(P2, c4, n, 252, w2.seed),
                                   1 << 20, 252, "Asian call K=100, 252 steps, 2^20 paths, "
                                   "d price / d (S0, v0, kappa, theta, xi, rho, r)", 1)
    return out


def cpu_baseline(target_s: float = 10.0):
    w, P, cs, threads, n = _oracle_sample(target_s)
    rate, dt = _time_oracle(w, P, cs, n)
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} of the {w.n_paths} paths x {w.n_steps} steps, 6 contracts, FP64 "
                      f"oracle on {threads} host threads ({dt:.1f} s)"}


def _workload_config(w, n, nc):
    """The workload's description, the same in both arms (what is computed, not
    how): the configuration is named by what it is, with its sizes."""
    return {"workload": w.name if n == w.n_paths else f"{w.name} (n_paths={n})",
            "n_paths": n, "n_steps": w.n_steps,
            "contracts": "European + Asian(M=252) calls, K in {90,100,110}",
            "estimates": 6 * nc, "truncation": "full", "rng": "philox4x32-10"}


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    per_step_s = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    w, P, cs, threads, n = _oracle_sample(per_step_s)
    for _ in range(args.warmup):
        _time_oracle(w, P, cs, n)
    times = []
    for _ in range(args.steps):
        _, dt = _time_oracle(w, P, cs, n)
        times.append(dt)
    step_s = statistics.mean(times)
    value = n * w.n_steps / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": _workload_config(w, w.n_paths, len(cs)),
        "sample": f"{n} of {w.n_paths} paths per timed step (value = sampled path-steps / time)",
        "precision": "fp64 oracle path and sums",
        "parallelism": f"{threads} host threads (OpenMP over fixed path chunks)",
        "greek_sets_per_s": 6.0 / step_s,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n} paths x {w.n_steps} steps per step, FP64 oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_2309_10477_gb300 import native as nv
    from paper_2309_10477_gb300 import workloads as wl

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = nv.load()
    stream = torch.cuda.current_stream()

    w = wl.multi_strike_fp32()
    nc = len(w.contracts)
    params = nv.make_params(**w.params)
    contracts = [nv.make_contract(*c) for c in w.contracts]
    opts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local)
    n = args.n_paths or w.n_paths
    path_begin = rank * n                       # weak scaling: one path range per rank
    n_tiles = -(-n // nv.HESTON_TILE_PATHS)
    rows = torch.empty(n_tiles * 12 * nc, dtype=torch.float64, device=dev)
    ws_bytes = nv.heston_mc_workspace_bytes(nc, n)
    ws = torch.empty(ws_bytes // 8, dtype=torch.float64, device=dev)
    out = torch.empty(nc * 12, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        nv.heston_mc_launch_tiles(params, contracts, path_begin, n, w.n_steps, w.seed, opts, rows)
        if ev is not None:
            ev[1].record(stream)
        nv.heston_mc_reduce_tiles(rows, n_tiles, nc, n, ws, ws_bytes, out, stream)
        if ev is not None:
            ev[2].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # measured issue rates of the pipes the kernels use: the roofline denominators
    from paper_2309_10477_gb300 import peaks as pipe_peaks
    pk = None
    t_pk = (time.time(), time.time())
    if not args.no_peaks:
        clocks.mark(True)
        t_pk = time.time()
        pk = pipe_peaks.measure(args.peak_seconds, local)
        t_pk = (t_pk, time.time())
        clocks.mark(False)

    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    clocks.mark(True)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)                    # evict L2 between timed steps (outside events)
        step(events[i])
    barrier()
    clocks.mark(False)
    step_ms = [e[0].elapsed_time(e[2]) for e in events]
    k1_ms = [e[0].elapsed_time(e[1]) for e in events]
    local_ms = statistics.mean(step_ms)
    local_k1 = statistics.mean(k1_ms)
    t = torch.tensor([local_ms, local_k1], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, k1 = float(t[0]), float(t[1])
    estimates = out.view(nc, 12).cpu().numpy()

    # one estimate split across the ranks (strong scaling next to the replica number):
    # each rank simulates its path range of the 2^22 paths, the tile rows are
    # all-gathered over NCCL and reduced in the fixed order -- all inside the timing
    sharded = None
    if world > 1 and not args.no_sharded:
        from paper_2309_10477_gb300 import parallel
        n_all = w.n_paths
        sopts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local)
        for _ in range(2):
            parallel.price_greeks_sharded(params, contracts, n_all, w.n_steps, w.seed, sopts)
        barrier()
        sh_times = []
        res_sh = None
        for i in range(max(3, min(args.steps, 20))):
            flush.fill_(i & 0xFF)
            barrier()
            t0 = time.perf_counter()
            res_sh = parallel.price_greeks_sharded(params, contracts, n_all, w.n_steps, w.seed, sopts)
            torch.cuda.synchronize()
            sh_times.append(time.perf_counter() - t0)
        tt = torch.tensor([statistics.mean(sh_times)], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        same = None
        if rank == 0:                          # the same estimate on this GPU alone
            ws_all_bytes = nv.heston_mc_workspace_bytes(nc, n_all)
            ws_all = torch.empty(ws_all_bytes // 8 + 32, dtype=torch.float64, device=dev)
            out_all = torch.empty(nc * 12, dtype=torch.float64, device=dev)
            nv.heston_mc_launch(params, contracts, n_all, w.n_steps, w.seed, sopts, ws_all,
                                ws_all_bytes, out_all)
            torch.cuda.synchronize()
            same = bool(torch.equal(out_all.view(nc, 12).cpu(), res_sh))
        barrier()
        sh_s = float(tt[0])
        sharded = {"workload": f"{w.name}: one estimate, the paths split across {world} ranks",
                   "scaling": "strong", "ms_per_estimate": sh_s * 1e3,
                   "path_steps_per_s": n_all * w.n_steps / sh_s,
                   "greek_sets_per_s": nc / sh_s,
                   "exchange": "NCCL all_gather of the 64-path tile rows, fixed-order reduction",
                   "identical_to_one_gpu": same,
                   "timing": "host clock around each estimate (launch, gather, reduce, result on the "
                             "host), barrier before each, max over ranks"}

    # config 1: one European call, 2^16 paths x 100 steps, FP64 path (FP64-pipe bound)
    fp64v = None
    if not args.no_fp64 and world == 1:
        w1 = wl.single_european_fp64()
        p1 = nv.make_params(**w1.params)
        c1 = [nv.make_contract(*c) for c in w1.contracts]
        ws1_bytes = nv.heston_mc_workspace_bytes(1, w1.n_paths)
        ws1 = torch.empty(ws1_bytes // 8 + 32, dtype=torch.float64, device=dev)
        out1 = torch.empty(12, dtype=torch.float64, device=dev)
        o1 = nv.make_options(prec=nv.HESTON_FP64, stream=stream, device=local)
        for _ in range(3):
            nv.heston_mc_launch(p1, c1, w1.n_paths, w1.n_steps, w1.seed, o1, ws1, ws1_bytes, out1)
        barrier()
        f_steps = max(5, min(args.steps, 50))
        fev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(f_steps)]
        clocks.mark(True)
        for i in range(f_steps):
            flush.fill_(i & 0xFF)
            fev[i][0].record(stream)
            nv.heston_mc_launch(p1, c1, w1.n_paths, w1.n_steps, w1.seed, o1, ws1, ws1_bytes, out1)
            fev[i][1].record(stream)
        barrier()
        clocks.mark(False)
        f_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in fev)
        est1 = out1.view(1, 12).cpu().numpy()[0]
        ps1 = w1.n_paths * w1.n_steps / (f_ms * 1e-3)
        # measured DFMA rate; without the micro-benchmarks, 2 FP64 FMAs per SM per clock
        dfma = (pk["dfma"]["thread_insts_per_s"] if pk else
                2.0 * torch.cuda.get_device_properties(dev).multi_processor_count * 2070e6)
        fp64v = {"workload": w1.name, "ms_per_step": f_ms, "path_steps_per_s": ps1,
                 "greek_sets_per_s": 1.0 / (f_ms * 1e-3), "gpu_launches_per_step": 3,
                 "estimates": dict(zip(nv.ESTIMATORS, est1[:6].tolist())),
                 "se": dict(zip(nv.ESTIMATORS, est1[6:].tolist())),
                 "roofline": {"bound": "fp64", "achieved": FP64_OPS_PER_PATH_STEP * ps1 / 1e12,
                              "peak": dfma / 1e12, "frac": FP64_OPS_PER_PATH_STEP * ps1 / dfma,
                              "unit": f"T FP64 operations/s ({FP64_OPS_PER_PATH_STEP} explicit FP64 "
                                      "operations per path-step; the FP64 log, sqrt, sin/cos and "
                                      "rsqrt run on the same pipe and are not counted; peak = the "
                                      "measured DFMA rate)"}}
        # from the committed ncu summary of this kernel (None once the device source changed)
        busy = _profile_value(FP64_PROFILE, r"sm__pipe_fp64_cycles_active \(of elapsed\)\*\* \| \*\*([0-9.]+) %")
        executed = _profile_value(FP64_PROFILE, r"DADD [0-9.]+: ([0-9.]+) arithmetic")
        fp64v["roofline"]["fp64_pipe_busy_ncu"] = None if busy is None else busy / 100.0
        fp64v["roofline"]["executed_fp64_per_path_step_ncu"] = executed
        if executed is not None:
            fp64v["roofline"]["frac_executed"] = executed * ps1 / dfma

    # randomised-QMC variant on the same workload: 32 replicates x 2^17 points
    qmc = None
    if not args.no_qmc and world == 1:
        R = 32
        tb_bytes = nv.heston_qmc_tables_bytes(w.n_steps)
        tables = torch.empty(tb_bytes // 8 + 1, dtype=torch.float64, device=dev)
        nv.heston_qmc_build_tables(w.n_steps, tables, tb_bytes, local)
        qws_bytes = nv.heston_mc_workspace_bytes_qmc(nc, n, w.n_steps, R)
        qws = torch.empty(qws_bytes // 8 + 1, dtype=torch.float64, device=dev)
        qout = torch.empty(nc * 12, dtype=torch.float64, device=dev)
        qopts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local,
                                rng=nv.HESTON_RNG_SOBOL_BB, n_shifts=R)
        for _ in range(3):
            nv.heston_mc_launch_qmc(params, contracts, n, w.n_steps, w.seed, qopts, tables, qws,
                                    qws_bytes, qout)
        barrier()
        q_steps = max(3, min(args.steps, 50))
        qev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(q_steps)]
        clocks.mark(True)
        for i in range(q_steps):
            flush.fill_(i & 0xFF)
            qev[i][0].record(stream)
            nv.heston_mc_launch_qmc(params, contracts, n, w.n_steps, w.seed, qopts, tables, qws,
                                    qws_bytes, qout)
            qev[i][1].record(stream)
        barrier()
        clocks.mark(False)
        q_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in qev)
        qest = qout.view(nc, 12).cpu().numpy()
        se_ratio = float(qest[1, 6] / estimates[1, 6])          # price SE, European K=100
        qmc = {"rng": f"sobol+brownian-bridge, {R} digital shifts x {n // R} points",
               "ms_per_step": q_ms, "path_steps_per_s": n * w.n_steps / (q_ms * 1e-3),
               "price_se_k100_euro": float(qest[1, 6]), "se_ratio_vs_philox": se_ratio,
               "path_steps_per_s_at_philox_se": n * w.n_steps / (q_ms * 1e-3) / se_ratio**2,
               "gpu_launches_per_step": 4}

    # scheme variants on the same workload and launch: Euler (Sec. 2.4.1) and QE
    schemes = None
    if not args.no_schemes and world == 1:
        schemes = {}
        # the paper's scheme as printed (Milstein, V floored at zero after each
        # update), Euler, and Andersen's QE, on the same workload and normals
        for sname, sid, strunc in (("milstein_paper_floor", nv.HESTON_SCHEME_MILSTEIN, nv.HESTON_TRUNC_PAPER_FLOOR),
                                   ("euler", nv.HESTON_SCHEME_EULER, nv.HESTON_TRUNC_FULL),
                                   ("qe", nv.HESTON_SCHEME_QE, nv.HESTON_TRUNC_FULL)):
            sopts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local, scheme=sid, trunc=strunc)
            sout = torch.empty(nc * 12, dtype=torch.float64, device=dev)

            def sstep():
                nv.heston_mc_launch(params, contracts, n, w.n_steps, w.seed, sopts, ws, ws_bytes, sout)

            for _ in range(3):
                sstep()
            barrier()
            s_steps = max(3, min(args.steps, 30))
            sev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(s_steps)]
            clocks.mark(True)
            for i in range(s_steps):
                flush.fill_(i & 0xFF)
                sev[i][0].record(stream)
                sstep()
                sev[i][1].record(stream)
            barrier()
            clocks.mark(False)
            s_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in sev)
            sest = sout.view(nc, 12).cpu().numpy()
            schemes[sname] = {"ms_per_step": s_ms, "path_steps_per_s": n * w.n_steps / (s_ms * 1e-3),
                              "price_k100_euro": float(sest[1, 0]), "price_se_k100_euro": float(sest[1, 6]),
                              "gpu_launches_per_step": 3}

    # batched form: 1024 uneven contracts in one persistent launch (captured in a
    # CUDA graph) against one launch per contract, same paths hence same SE
    batched = None
    if not args.no_batch and world == 1:
        from paper_2309_10477_gb300 import autotune
        bitems = [nv.make_batch_item(nv.make_params(**d["params"]), nv.make_contract(*d["contract"]),
                                     d["n_paths"], d["n_steps"], w.seed + 1000003 * i)
                  for i, d in enumerate(wl.batched_contracts(1024)[:args.batch_contracts])]
        bopts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local)
        plan = nv.heston_batch_plan_make(bitems, bopts)
        desc = torch.empty(plan.descriptor_bytes // 8 + 32, dtype=torch.float64, device=dev)
        bws = torch.empty(plan.workspace_bytes // 8 + 32, dtype=torch.float64, device=dev)
        bout = torch.empty(len(bitems) * 12, dtype=torch.float64, device=dev)
        nv.heston_batch_prepare(bitems, bopts, plan, desc)
        (blk, grd), tune_ms = autotune.tune_batch(plan, desc, bws, bout, bopts, stream=stream)
        topts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local,
                                block_threads=blk, grid_ctas=grd)
        gstream = torch.cuda.Stream(device=dev)
        gstream.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gstream):
            gopts = nv.make_options(prec=nv.HESTON_FP32, stream=torch.cuda.current_stream(),
                                    device=local, block_threads=blk, grid_ctas=grd)
            nv.heston_mc_launch_batch(plan, desc, gopts, bws, bout)
        graph.replay()
        barrier()
        b_steps = max(3, min(args.steps // 20, 10))
        clocks.mark(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(b_steps):
            graph.replay()
        e1.record(stream)
        barrier()
        batch_ms = e0.elapsed_time(e1) / b_steps
        # one launch per contract, each with its own workspace slice, back to back
        single = []
        for it in bitems:
            sb = nv.heston_mc_workspace_bytes(1, it.n_paths)
            single.append((it, sb))
        sws = torch.empty(max(sb for _, sb in single) // 8 + 32, dtype=torch.float64, device=dev)
        sout = torch.empty(len(bitems) * 12, dtype=torch.float64, device=dev)
        def per_contract():
            for i, (it, sb) in enumerate(single):
                nv.heston_mc_launch(it.params, [it.contract], it.n_paths, it.n_steps, it.rng_seed,
                                    bopts, sws, sb, sout[i * 12:(i + 1) * 12])
        per_contract()
        barrier()
        e0.record(stream)
        for _ in range(2):
            per_contract()
        e1.record(stream)
        barrier()
        clocks.mark(False)
        single_ms = e0.elapsed_time(e1) / 2
        same = bool(torch.equal(torch.nan_to_num(bout), torch.nan_to_num(sout)))
        n_unstable = int((~torch.isfinite(bout.view(-1, 12)[:, [3, 5, 9, 11]])).any(dim=1).sum())
        # roofline of the persistent kernel: the method's issue slots per path-step (92
        # with an Asian date every step, 88 without), and the kernel's own minimum (64
        # with a date every step, 3.5 fewer without: ex2 + 5 FP32 packed two per slot)
        def date_frac(it):
            return (min(it.contract.n_monitor or it.n_steps, it.n_steps) / it.n_steps
                    if it.contract.payoff == nv.HESTON_ASIAN_ARITH else 0.0)
        slots = sum(it.n_paths * it.n_steps * (METHOD_SLOTS_NO_DATE + (METHOD_SLOTS_PER_PATH_STEP
                                                                      - METHOD_SLOTS_NO_DATE) * date_frac(it))
                    for it in bitems)
        slots_kernel = sum(it.n_paths * it.n_steps * (BATCH_SLOTS_PER_PATH_STEP - 3.5 * (1.0 - date_frac(it)))
                           for it in bitems)
        n_sm_b = torch.cuda.get_device_properties(dev).multi_processor_count
        max_mhz_b = float(_measured_peaks().get("sm_max_mhz") or 2070.0)
        # the measured issue rate (FFMA micro-benchmark), else SMs x 128 lanes x max clock
        peak_b = (max(v["thread_insts_per_s"] for k_, v in pk.items() if not k_.endswith("_mix")) / 1e12 if pk
                  else n_sm_b * ISSUE_LANES_PER_SM_CLK * max_mhz_b * 1e6 / 1e12)
        ach_b = slots / (batch_ms * 1e-3) / 1e12
        ach_bk = slots_kernel / (batch_ms * 1e-3) / 1e12
        batched = {"workload": f"{len(bitems)} seeded uneven contracts: K~U[70,130], T in {{0.25,0.5,1,2}}, "
                               "paths 2^U (U~U[14,20]), steps 50..500, European/Asian 50/50, FP32",
                   "total_path_steps": int(plan.total_path_steps),
                   "batch_ms": batch_ms, "greek_sets_per_s": len(bitems) / (batch_ms * 1e-3),
                   "path_steps_per_s": plan.total_path_steps / (batch_ms * 1e-3),
                   "per_contract_ms": single_ms,
                   "per_contract_greek_sets_per_s": len(bitems) / (single_ms * 1e-3),
                   "speedup_vs_per_contract": single_ms / batch_ms,
                   "results_identical_to_per_contract": same,
                   "contracts_with_unstable_vega_theta": n_unstable,
                   "launch_shape": {"block_threads": blk, "grid_ctas": grd,
                                    "tuned_candidates": len(tune_ms)},
                   "graph": "memset + persistent kernel + 2 reductions captured, replayed",
                   "roofline": {"bound": "alu", "kernel": "heston_batch_kernel<FULL> (graph replay)",
                                "achieved": ach_b, "peak": peak_b,
                                "unit": "T issue slots/s (92 per path-step with an Asian date every "
                                        "step, 88 without; peak: the measured issue rate, as for "
                                        "the path kernel)",
                                "frac": ach_b / peak_b,
                                "kernel_slot_model": {"slots_per_path_step": "64 with an Asian date "
                                                      "every step, 60.5 without",
                                                      "achieved": ach_bk, "frac": ach_bk / peak_b}}}

    # adjoint gradient: 252-step Asian call, 2^20 paths, d price / d (S0, v0, kappa, theta, xi, rho, r)
    adjoint = None
    if not args.no_adjoint and world == 1:
        an, aN = 1 << 20, 252
        ac = nv.make_contract(1, 100.0, 1.0)
        aws_bytes = nv.heston_adjoint_workspace_bytes(an, aN)
        aws = torch.empty(aws_bytes // 8 + 32, dtype=torch.float64, device=dev)
        aprice = torch.empty(2, dtype=torch.float64, device=dev)
        agrad = torch.empty(14, dtype=torch.float64, device=dev)
        aopts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local)
        for _ in range(2):
            nv.heston_mc_adjoint_forward(params, ac, an, aN, w.seed, aopts, aws, aws_bytes, aprice)
            nv.heston_mc_adjoint_backward(params, ac, an, aN, w.seed, aopts, aws, aws_bytes, agrad)
        barrier()
        a_steps = 5
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd, bwd = [], []
        clocks.mark(True)
        for _ in range(a_steps):
            ev[0].record(stream)
            nv.heston_mc_adjoint_forward(params, ac, an, aN, w.seed, aopts, aws, aws_bytes, aprice)
            ev[1].record(stream)
            nv.heston_mc_adjoint_backward(params, ac, an, aN, w.seed, aopts, aws, aws_bytes, agrad)
            ev[2].record(stream)
            ev[2].synchronize()
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[1].elapsed_time(ev[2]))
        clocks.mark(False)
        gv = agrad.cpu().numpy()
        adjoint = {"workload": "Asian call K=100, 252 dates/steps, 2^20 paths, FP32 path / FP64 sums",
                   "forward_ms": statistics.mean(fwd), "backward_ms": statistics.mean(bwd),
                   "checkpoint_every_steps": 8,
                   "price": float(aprice[0]), "gradient": dict(zip(
                       ("S0", "v0", "kappa", "theta", "xi", "rho", "r"), gv[:7].tolist())),
                   "gradient_se": gv[7:].tolist()}

    # serving: Poisson arrivals of single-contract requests into the native
    # continuous-batching engine; latency is submit -> result on the host
    serving = None
    if not args.no_serve and world == 1:
        import numpy as np
        rate, dur = args.serve_rate, args.serve_seconds
        g = np.random.Generator(np.random.PCG64(2309))
        n_req = int(rate * dur)
        arrivals = np.cumsum(g.exponential(1.0 / rate, n_req))
        reqs = [nv.make_batch_item(nv.make_params(**d["params"]), nv.make_contract(*d["contract"]),
                                   d["n_paths"], d["n_steps"], w.seed + 7919 * i)
                for i, d in enumerate(wl.serving_requests(n_req, seed=2309))]
        req_path_steps = sum(it.n_paths * it.n_steps for it in reqs)
        srv = nv.HestonServer(1 << 30, tiles_per_round=args.serve_tiles_per_round, device=local)
        for t in [srv.submit(it) for it in reqs[:64]]:           # warm-up
            srv.wait(t, 60000)
        tickets = [0] * n_req
        lat = [0.0] * n_req
        queued_max = [0]
        submitted = threading.Event()

        def consume():
            for i in range(n_req):
                while tickets[i] == 0:
                    time.sleep(0.0002)
                r = srv.wait(tickets[i], 120000)
                assert r is not None and r[0].status >= 0
                lat[i] = r[1]

        def watch():
            while not submitted.is_set():
                st = srv.stats()
                queued_max[0] = max(queued_max[0], st.queued + st.active)
                time.sleep(0.01)

        th_c, th_w = threading.Thread(target=consume), threading.Thread(target=watch)
        st0 = srv.stats()
        clocks.mark(True)
        th_c.start()
        th_w.start()
        t0 = time.perf_counter()
        for i in range(n_req):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            tickets[i] = srv.submit(reqs[i])
        submit_s = time.perf_counter() - t0
        st_mid = srv.stats()
        submitted.set()
        th_w.join()
        # the largest of the 10 ms samples and the count at the last arrival
        queued_max[0] = max(queued_max[0], int(st_mid.queued + st_mid.active))
        th_c.join()
        wall_s = time.perf_counter() - t0
        clocks.mark(False)
        st1 = srv.stats()
        # capacity: 2000 requests of the same stream submitted at once, against the
        # same requests launched one per contract (same paths, hence the same SE)
        creqs = [nv.make_batch_item(nv.make_params(**d["params"]), nv.make_contract(*d["contract"]),
                                    d["n_paths"], d["n_steps"], w.seed + 104729 * i)
                 for i, d in enumerate(wl.serving_requests(2000, seed=77))]
        torch.cuda.synchronize()
        t_c = time.perf_counter()
        ctk = [srv.submit(it) for it in creqs]
        cres = [srv.wait(t, 120000) for t in ctk]
        cap_s = time.perf_counter() - t_c
        srv.close()
        max_np = max(it.n_paths for it in creqs)
        cws_bytes = nv.heston_mc_workspace_bytes(1, max_np)
        cws = torch.empty(cws_bytes // 8 + 32, dtype=torch.float64, device=dev)
        cout = torch.empty(len(creqs) * 12, dtype=torch.float64, device=dev)
        copts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, it in enumerate(creqs):
            nv.heston_mc_launch(it.params, [it.contract], it.n_paths, it.n_steps, it.rng_seed, copts,
                                cws, nv.heston_mc_workspace_bytes(1, it.n_paths), cout[i * 12:(i + 1) * 12])
        e1.record(stream)
        e1.synchronize()
        pc_s = e0.elapsed_time(e1) * 1e-3
        cgot = np.array([[getattr(r, k) for k in nv.ESTIMATORS] + list(r.se) for r, _ in cres])
        csame = bool(np.array_equal(np.nan_to_num(cgot), np.nan_to_num(cout.view(-1, 12).cpu().numpy())))
        la = np.array(lat) * 1e3
        # percentiles after a warm-up of 5 s (or a twelfth of a shorter run)
        warm_s = min(5.0, dur / 12.0)
        la_w = la[np.asarray(arrivals) >= warm_s]
        serving = {"workload": f"Poisson arrivals at {rate:.0f}/s for {dur:.0f} s ({n_req} requests), "
                               "each one contract with parameters drawn like the batched form, "
                               "paths 2^U (U~U[16,22]), steps 50..252, European/Asian, FP32",
                   "offered_load_vs_batched_kernel": None,
                   "offered_path_steps_per_s": req_path_steps / arrivals[-1],
                   "latency_ms": {"p50": float(np.percentile(la_w, 50)), "p90": float(np.percentile(la_w, 90)),
                                  "p99": float(np.percentile(la_w, 99)), "max": float(la_w.max()),
                                  "over": f"requests submitted {warm_s:.0f} s or later ({la_w.size})"},
                   "latency_ms_all_requests": {"p50": float(np.percentile(la, 50)),
                                               "p99": float(np.percentile(la, 99)), "max": float(la.max())},
                   "greek_sets_per_s": n_req / wall_s, "path_steps_per_s": req_path_steps / wall_s,
                   "drain_after_last_arrival_ms": (wall_s - submit_s) * 1e3,
                   "max_requests_in_system": queued_max[0],
                   "in_system_at_last_arrival": int(st_mid.queued + st_mid.active),
                   "rounds": int(st1.rounds - st0.rounds),
                   "tiles_per_round": args.serve_tiles_per_round,
                   "memory_peak_bytes": int(st1.memory_peak),
                   "saturated": {"requests": len(creqs), "greek_sets_per_s": len(creqs) / cap_s,
                                 "per_contract_greek_sets_per_s": len(creqs) / pc_s,
                                 "speedup_vs_per_contract": pc_s / cap_s,
                                 "results_identical_to_per_contract": csame,
                                 "note": "served: host wall time from first submit to last result; "
                                         "per-contract: CUDA events around 2000 heston_mc_launch calls"}}
        if batched is not None:
            serving["offered_load_vs_batched_kernel"] = (serving["offered_path_steps_per_s"]
                                                         / batched["path_steps_per_s"])

    # end to end through the synchronous host API (host structs in, results out)
    res_arr = (nv.heston_result * nc)()
    carr = (nv.heston_contract * nc)(*contracts)
    e2e_opts = nv.make_options(prec=nv.HESTON_FP32, stream=stream, device=local)
    for _ in range(2):
        lib.heston_mc_price_greeks_ex(ctypes.byref(params), carr, nc, n, w.n_steps, w.seed,
                                      ctypes.byref(e2e_opts), res_arr)
    barrier()
    clocks.mark(True)
    e2e_steps = max(3, min(args.steps, 20))
    e2e_times = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        rc = lib.heston_mc_price_greeks_ex(ctypes.byref(params), carr, nc, n, w.n_steps, w.seed,
                                           ctypes.byref(e2e_opts), res_arr)
        e2e_times.append(time.perf_counter() - t0)
        assert rc >= 0, nv.heston_status_string(rc)
    clocks.mark(False)
    clocks.stop()
    e2e_s = torch.tensor([statistics.mean(e2e_times)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(e2e_s, op=dist.ReduceOp.MAX)

    path_steps = n * w.n_steps
    value = world * path_steps / (ms * 1e-3)
    if rank == 0:
        peaks = _measured_peaks()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        clk = clocks.summary()
        max_mhz = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
        nominal_tinst = n_sm * ISSUE_LANES_PER_SM_CLK * max_mhz * 1e6 / 1e12
        # measured: the FP32 FMA rate, one thread-instruction per lane per clock, the
        # highest rate any instruction kind reaches (the machine's issue rate)
        peak_tinst = (max(v["thread_insts_per_s"] for k_, v in pk.items() if not k_.endswith("_mix")) / 1e12 if pk
                      else nominal_tinst)
        achieved_tinst = path_steps * METHOD_SLOTS_PER_PATH_STEP / (k1 * 1e-3) / 1e12
        achieved_kernel = path_steps * ALGO_SLOTS_PER_PATH_STEP / (k1 * 1e-3) / 1e12
        pk_clk = clocks.summary_between(*t_pk)
        pk_mhz = pk_clk.get("sm_mhz") or max_mhz
        traffic = _profiled_traffic()
        mix_ceiling = (None if not pk or "heavy_mix" not in pk else
                       pk["heavy_mix"]["thread_insts_per_s"] / MIX_INSTS_PER_UNIT * MIX_PATH_STEPS_PER_UNIT)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": _workload_config(w, n, nc),
            "precision": "fp32 path, fp64 sums", "parallelism": f"dp{world} (path ranges)",
            "l2": "flushed between timed steps (256 MiB write outside the events)",
            "greek_sets_per_s": world * nc / (ms * 1e-3),
            "price_se_k100_euro": float(estimates[1, 6]),
            "fixed_se_note": "SE target = the FP64 oracle's SE on the same normals; the GPU SE "
                             "matches it to 1e-3 (tested), so time-to-target = time per step",
            "e2e": {"value": world * path_steps / float(e2e_s[0]), "unit": UNIT,
                    "h2d_bytes_per_step": ctypes.sizeof(nv.heston_params)
                    + nc * ctypes.sizeof(nv.heston_contract),
                    "d2h_bytes_per_step": nc * 12 * 8},
            "gpu_launches": 3 * args.steps * world,         # path kernel + 2 reductions per step, all ranks
            "roofline": {"bound": "alu", "kernel": "heston_paths_kernel<float,FULL,ASIAN>",
                         "achieved": achieved_tinst, "peak": peak_tinst,
                         "unit": f"T issue slots/s ({METHOD_SLOTS_PER_PATH_STEP} algorithmic issue slots per "
                                 "path-step, one per operation the method computes: ~45 INT32 (Philox) "
                                 "+ ~41 FP32 + 6 MUFU; peak = the measured issue rate, the FP32 FMA "
                                 "micro-benchmark's thread-instructions/s)",
                         "peak_source": ("measured (pipe_peaks, this run)" if pk else
                                         "nominal: SMs x 128 lanes x max clock (--no-peaks)"),
                         "nominal_peak": nominal_tinst,
                         "frac": achieved_tinst / peak_tinst,
                         "kernel_slot_model": {
                             "slots_per_path_step": ALGO_SLOTS_PER_PATH_STEP,
                             "ops_per_path_step": ALGO_OPS_PER_PATH_STEP,
                             "note": "the path kernel's own minimum: FP32 operations packed two per "
                                     "f32x2 instruction, Philox's warp-uniform products from a per-warp "
                                     "table and its per-path second-round product hoisted out of the loop",
                             "achieved": achieved_kernel, "frac": achieved_kernel / peak_tinst,
                             "ops_per_s": path_steps * ALGO_OPS_PER_PATH_STEP / (k1 * 1e-3) / 1e12},
                         "traffic": traffic,
                         "binding_pipe": {
                             "pipe": "fmaheavy (the FMA pipe's heavy half)",
                             "busy_ncu": (None if (hb := _profile_value(
                                 PROFILE_SUMMARY, r"sm__pipe_fmaheavy_cycles_active \(of elapsed\) \| \*\*([0-9.]+) %"))
                                 is None else hb / 100.0),
                             "model": "per warp and lane-step (64 path-steps): 15 Philox wide multiplies x 4 "
                                      "heavy-pipe cycles + 44 f32x2 FMA-pipe instructions x 2 = 148 cycles",
                             "ceiling_path_steps_per_s": HEAVY_LANE_STEP_PATHS * 4 * n_sm
                             * (pk_mhz or max_mhz) * 1e6 / HEAVY_CYCLES_PER_LANE_STEP,
                             "frac": (path_steps / (k1 * 1e-3)) / (HEAVY_LANE_STEP_PATHS * 4 * n_sm
                                                                  * (pk_mhz or max_mhz) * 1e6
                                                                  / HEAVY_CYCLES_PER_LANE_STEP),
                             "ceiling_measured_path_steps_per_s": mix_ceiling,
                             "frac_measured": (None if mix_ceiling is None
                                               else (path_steps / (k1 * 1e-3)) / mix_ceiling),
                             "measured_by": "heavy_mix micro-benchmark (15 wide multiplies + 44 f32x2 "
                                            "FMAs per lane and step, independent chains, this run)"},
                         "kernel_ms": k1,
                         "path_steps_per_s_kernel": path_steps / (k1 * 1e-3)},
            "pipe_peaks": None if pk is None else {
                "unit": "T thread-instructions/s", "sm_mhz_median": pk_mhz,
                "rates": {k: v["thread_insts_per_s"] / 1e12 for k, v in pk.items()},
                "per_sm_per_clock": {k: v["thread_insts_per_s"] / (n_sm * pk_mhz * 1e6)
                                     for k, v in pk.items()}},
            "clocks": clk,
        }
        if fp64v is not None:
            line["fp64_single_european_variant"] = fp64v
        if sharded is not None:
            line["sharded_variant"] = sharded
        if qmc is not None:
            line["qmc_variant"] = qmc
        if batched is not None:
            line["batched_variant"] = batched
        if adjoint is not None:
            line["adjoint_variant"] = adjoint
        if serving is not None:
            line["serving_variant"] = serving
        if schemes is not None:
            line["scheme_variants"] = schemes
        if not args.no_cpu_baseline and world == 1:      # the oracle baseline: rank 0 at N = 1 only
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
            line["cpu_baseline"]["host"] = host_info()
            line["cpu_baselines_by_config"] = cpu_baselines(args.cpu_config_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-qmc", action="store_true", help="skip the quasi-Monte Carlo variant")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 1024-contract form")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint gradient")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-schemes", action="store_true", help="skip the Euler / QE variants")
    ap.add_argument("--batch-contracts", type=int, default=1024,
                    help="contracts in the batched mix (the first n of the seeded 1024)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="request arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-tiles-per-round", type=int, default=65536)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-config-seconds", type=float, default=2.0,
                    help="oracle seconds per configuration and core mode")
    ap.add_argument("--peak-seconds", type=float, default=0.3,
                    help="timed seconds per instruction kind of the pipe micro-benchmarks")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 single-European variant")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the pipe micro-benchmarks (roofline against the nominal peak; for ncu runs)")
    ap.add_argument("--no-sharded", action="store_true",
                    help="skip the estimate split across ranks (N > 1)")
    ap.add_argument("--n-paths", type=int, default=0,
                    help="paths per rank (default: the workload's 2^22); small cases for ncu")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
