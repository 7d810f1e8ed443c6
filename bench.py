"""Benchmark of the constraint-aware auto-tuning hot path on B300.

Workload (default): the large space — 16 integer parameters, 51,609,600,000 Cartesian points
(int64 index), 12 constraints, 695,228,960 valid configurations as packed uint64 keys.  One step
is the whole hot path of a tuning session on it, from a fresh definition: define_space from the
host value lists and constraints, the space's first build_valid_space (decode, predicates,
compaction into the sorted key array), then generations 0 and 1 of constraint-aware DE at pop 256
(initial valid sample, mutation + crossover, validity lookup, exhaustive-equivalent Hamming
repair, fitness lookup in a seeded lognormal table, greedy selection).

Headline `value`: valid configurations enumerated per second (all ranks' |V| per step / step
time, CUDA events on the launching stream).  `e2e`: the same step through the public C-ABI with
the population, fitness and best read back to pinned host buffers, host wall clock.  `also`: the
metric's other parts (repaired candidates/s on the large space, batched runs/s and their ratio to
the same runs done one at a time) and the rebuild of an already built space.  `--full` adds every
sub-metric on an earlier stdout line; the headline is always the last line.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--full]
Under torchrun each rank runs an independent replica (weak scaling).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "valid configs enumerated/s; repaired candidates/s; batched runs/s vs plain"
UNIT = "valid configs/s"
L2_BYTES = 126 * 2 ** 20
POP = 256
CONFIG = {"workload": "large: 16 int params, 51,609,600,000 Cartesian points, 12 constraints, 695,228,960 valid; "
                      "step = first build: define_space from host lists + the space's first build_valid_space "
                      "(tables, every level's count, scan, size read-back and emit) + DE generations 0 (initial "
                      "sample) and 1 (pop 256) + destroy",
          "pop": POP, "l2": "working set 5.6 GB of keys > 126 MB L2 (no flush needed)"}


HOST_WARM_S = 1.0   # seconds of continuous host work before a timed region


def host_warm(seconds=None):
    """Busy host for `seconds`: the GPU machines' virtual CPUs slow down while idle (see the
    warm-up note in run_ours), and host-bound timings must not start on a cold CPU."""
    seconds = HOST_WARM_S if seconds is None else seconds
    t = time.perf_counter()
    while time.perf_counter() - t < seconds:
        pass


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except FileNotFoundError:
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.t.join(timeout=2)

    def summary(self, t0, t1):
        rows = [s for t, s in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or [s for _, s in self.samples]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# oracle baseline (host cores; the oracle as it stands)
# ------------------------------------------------------------------------------------------
def oracle_windows(n_windows, width, offset_seed=0):
    from paper_2606_28372_b300 import workloads as W
    cart = W.large_space().cartesian_size
    step = cart // n_windows
    rng = np.random.default_rng(offset_seed)
    return [(i * step + int(rng.integers(0, step - width)), width) for i in range(n_windows)]


_ORACLE_SPACE = None


def time_oracle(windows):
    global _ORACLE_SPACE
    from oracle import oracle as O
    from paper_2606_28372_b300 import workloads as W
    if _ORACLE_SPACE is None:                      # parsed once per process
        _ORACLE_SPACE = O.from_def(W.large_space())
    sp = _ORACLE_SPACE
    t0 = time.perf_counter()
    found = 0
    for c0, w in windows:
        found += O.enumerate_range(sp, c0, c0 + w, count_only=False).size
    dt = time.perf_counter() - t0
    return found, dt


def _oracle_window_worker(windows):
    """One process of the multi-core baseline: the oracle, as it stands, on its share of windows."""
    found, dt = time_oracle(windows)
    return found, dt


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(seconds_target=12.0):
    """The oracle, as it stands, on every host core: windows of the large space's Cartesian
    range spread over a process pool (started with spawn, so no process inherits CUDA state),
    timed end to end; the single-thread rate of the same windows is reported beside it."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    wins = oracle_windows(512, 1_000_000, offset_seed=1)
    spread = wins[:: len(wins) // 8][:8]             # single thread, windows over the whole range
    found1, dt1 = time_oracle(spread)
    single = found1 / dt1
    per_window = dt1 / len(spread)
    n = max(cores, min(len(wins), int(cores * seconds_target / max(per_window, 1e-3))))
    n -= n % cores
    sample = [wins[i * len(wins) // n] for i in range(n)]   # spread over the whole range
    shares = [sample[i::cores] for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_window_worker, [[w] for w in wins[:cores]])   # start-up and imports, untimed
        t0 = time.perf_counter()
        res = pool.map(_oracle_window_worker, shares)
        wall = time.perf_counter() - t0
    found = sum(r[0] for r in res)
    return {"value": found / wall, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "single_thread_value": single,
            "sample": f"brute-force enumeration of {n} windows x 1e6 Cartesian indices spread evenly over the "
                      f"large space, {n // cores} per process on {cores} processes ({found} valid found in "
                      f"{wall:.1f} s wall); single thread on 8 of the windows: {single:.0f} valid/s"}


# ------------------------------------------------------------------------------------------
# distributed plumbing
# ------------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(ms, dist, dev=None):
    """The slowest rank's time (the job's time): all-reduce MAX over the process group."""
    if not dist:
        return ms
    import torch
    tt = torch.tensor([ms], dtype=torch.float64, device=dev if dev is not None else "cpu")
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(units_per_rank_step, world, steps, ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank_step * steps / (ms / 1000.0)


REF_WINDOWS_PER_PROC, REF_WINDOW = 8, 31_250   # per process and step: 250,000 Cartesian indices


def run_reference(args):
    """The reference arm: the oracle, as it stands, on every host core (a spawn-started process
    pool; per process and step, 8 windows of 31,250 Cartesian indices, the windows of a step
    spread over the whole large space, so that every step meets some valid blocks), the same
    metric and workload as our arm."""
    import multiprocessing as mp
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    n_steps = args.steps + args.warmup
    per = REF_WINDOWS_PER_PROC
    wins = oracle_windows(cores * per * n_steps, REF_WINDOW, offset_seed=2)
    step_wins = [wins[s::n_steps] for s in range(n_steps)]   # each step: cores x per windows over the range
    ctx = mp.get_context("spawn")
    times, found = [], 0
    with ctx.Pool(cores) as pool:
        for s in range(n_steps):
            shares = [step_wins[s][c::cores] for c in range(cores)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_window_worker, shares)
            dt = time.perf_counter() - t0
            if s >= args.warmup:
                times.append(dt)
                found += sum(r[0] for r in res)
    total = sum(times)
    v = found / total
    sample = (f"{args.steps} steps x {cores} processes x {per} windows x {REF_WINDOW:,} Cartesian indices spread "
              f"over the large space ({found} valid found), brute-force oracle enumeration on {cores} processes "
              f"({cpu_model()})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": dict(CONFIG, parallelism=f"replicas x{world}"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def traffic_from_profile():
    """Per-launch DRAM bytes of the emit kernel from the committed ncu summary, if the kernel's
    source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "expand_emit_large.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_key:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not (m and h):
        return None
    if kernel_source_hash("k_pemit") != h.group(1)[:16]:
        return None
    return float(m.group(1))


def kernel_source_hash(name):
    """First 16 hex digits of the SHA-256 of a kernel's definition in space.cu (from its
    `__global__` line to the closing brace at the start of a line)."""
    src = open(os.path.join(ROOT, "paper_2606_28372_b300", "csrc", "space.cu")).read()
    m = re.search(r"^__global__[^{;]*?\b" + name + r"\(", src, re.M | re.S)
    if not m:
        return None
    end = src.index("\n}\n", m.start()) + 3
    return hashlib.sha256(src[m.start():end].encode()).hexdigest()[:16]


def first_build_step(ct, sd, table, rank, emit):
    """One step of the headline: a tuning session's device work from a fresh definition.
    ct_define_space from the host lists, the first ct_build_valid_space of that space (device
    upload of the descriptor, the compact, truth-mask and pattern tables, every level's count,
    scan and emit with its size read back), the fitness table attached, a DE run created and its
    generations 0 (initial sample) and 1 (pop 256) launched, then both handles destroyed (their
    blocks go back to the library's cache in stream order).  `emit` collects the last-level
    emit's CUDA-event time and algorithmic bytes."""
    s = ct.Space.from_def(sd)
    s.set_timing(True)
    s.build()
    s.set_fitness(table)
    o = ct.Opt(s, "de", POP, seed=rank)
    o.step(0)
    o.step(1)
    st = s.build_stats()
    last = st["levels"] - 1
    emit.append((st["emit_ms"][last], 8 * st["children"][last] + 8 * st["parents"][last], st["children"][last]))
    del o, s


def timed_loop(torch, ct, step, steps, warmup, stream, dist):
    """W warm-up steps (more until the host has been busy for HOST_WARM_S), then exactly `steps`
    steps between CUDA events on the launching stream, a barrier and a synchronisation on both
    sides.  Returns (device ms over the timed steps, wall t0, wall t1, the library's kernel
    launches inside the timed region)."""
    tw = time.perf_counter()
    done = 0
    while done < warmup or time.perf_counter() - tw < HOST_WARM_S:
        step(False)
        done += 1
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    l0 = ct.launch_count()
    e0.record(stream)
    for _ in range(steps):
        step(True)
    e1.record(stream)
    launches = ct.launch_count() - l0
    torch.cuda.synchronize()
    t1 = time.time()
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1), t0, t1, launches


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sd = W.SPACES[args.workload]()

    # ---- input synthesis (untimed): the fitness table over the valid ranks ----
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    g = torch.Generator(device=dev)
    g.manual_seed(1234 + rank)
    table = torch.exp(torch.randn(nv, generator=g, device=dev, dtype=torch.float32))

    # ---- headline: first builds of freshly defined spaces + DE generations 0 and 1 ----
    # The host CPUs of the GPU machines run several times slower after an idle spell and take
    # about a second of continuous work to come back to speed; the warm-up keeps the host busy
    # for at least HOST_WARM_S so that the timed region does not time the host's wake-up.  The
    # clock sampler starts first so that it is already sampling when the timed region begins.
    clocks = ClockSampler(local)
    clocks.start()
    emit = []
    ms, t0, t1, launches = timed_loop(torch, ct, lambda rec: first_build_step(ct, sd, table, rank, emit if rec else []),
                                      args.steps, args.warmup, stream, dist)
    ms = max_over_ranks(ms, dist, dev)
    time.sleep(0.2)
    clocks.stop()
    ms_step = ms / args.steps
    value = job_throughput(nv, world, args.steps, ms)

    # ---- roofline of the dominant kernel (last-level pattern emit), from the timed steps ----
    hbm, peak_kind = peaks()
    emit_avg_ms = float(np.mean([e[0] for e in emit]))
    emit_bytes = float(np.mean([e[1] for e in emit]))
    achieved = emit_bytes / (emit_avg_ms / 1000.0) / 1e9
    tpk = traffic_from_profile()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": (tpk * emit[-1][2]) if tpk else None,
                "traffic_source": "not measured in this run: ncu DRAM bytes per key of the same kernel source "
                                  "(profiles/expand_emit_large.md, 146M-key slice) x keys written per launch"
                                  if tpk else "null: no ncu capture of the current kernel source",
                "kernel": "k_pemit, last level of a first build_valid_space",
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": emit_bytes, "avg_launch_ms": emit_avg_ms,
                "share_of_step": emit_avg_ms / ms_step}

    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "ms_per_step": ms_step, "roofline": roofline, "gpu_launches": launches,
                              "clocks": clocks.summary(t0, t1), "quick": True}), flush=True)
        return 0

    # ---- rebuild of an already built space (labelled sub-metric, not the headline) ----
    sp.set_fitness(table)
    opt = ct.Opt(sp, "de", POP, seed=rank)

    def rebuild_step(rec):
        sp.build()
        opt.run_graph(0, 2)   # DE generations 0 and 1, one CUDA graph (dropped if a build moves the keys)

    rb_ms, _, _, _ = timed_loop(torch, ct, rebuild_step, args.steps, args.warmup, stream, dist)
    rb_ms = max_over_ranks(rb_ms, dist, dev)
    hinted = bool(sp.build_stats()["hinted"])
    del opt

    # ---- end to end through the C-ABI with host buffers ----
    keys_h = torch.empty(POP, dtype=torch.int64, pin_memory=True)     # the caller's host result buffers
    fit_h = torch.empty(POP, dtype=torch.float32, pin_memory=True)
    kd = torch.empty(POP, dtype=torch.int64, device=dev)
    fd = torch.empty(POP, dtype=torch.float32, device=dev)
    phases = {k: [] for k in ("define", "build", "create", "generations", "read_back", "destroy")}

    def e2e_step(record=False):
        t = [time.perf_counter()]
        s2 = ct.Space.from_def(sd)              # host lists -> library (H2D of the definition)
        t.append(time.perf_counter())
        n2 = s2.build()                          # D2H of |V|
        t.append(time.perf_counter())
        s2.set_fitness(table)
        o2 = ct.Opt(s2, "de", POP, seed=rank)
        t.append(time.perf_counter())
        o2.step(0)
        o2.step(1)
        t.append(time.perf_counter())
        o2.state(kd, fd)
        keys_h.copy_(kd, non_blocking=True)
        fit_h.copy_(fd, non_blocking=True)
        b = o2.best()                            # syncs
        t.append(time.perf_counter())
        del o2, s2
        t.append(time.perf_counter())
        if record:
            for k, a, z in zip(phases, t, t[1:]):
                phases[k].append(1000 * (z - a))
        return n2, b

    h2d = sum(8 * len(v) + 4 for v in sd.values) + 16 * sum(len(c) for c in sd.constraints)
    d2h = 8 + POP * 12 + 8 + 4 + 8 + 16
    tw = time.perf_counter()                    # untimed: at least one step, host back to speed
    while True:
        e2e_step()
        if time.perf_counter() - tw >= HOST_WARM_S:
            break
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 10))
    ta = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step(record=True)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - ta) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e = {"value": world * nv / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": 1000 * e2e_s,
           "note": "host wall clock: the headline step plus population, fitness and best read back to pinned host buffers",
           "phase_ms_median": {k: round(float(np.median(v)), 4) for k, v in phases.items()}}

    # ---- the metric's other two parts, compact ----
    also = {"rebuild_ms_per_step": rb_ms / args.steps, "rebuild_valid_configs_per_s": job_throughput(nv, world, args.steps, rb_ms),
            "rebuild_note": "build of an already built space (levels launched from its previous sizes) + DE gens 0-1 as one graph",
            "rebuild_hinted": hinted}
    rr = repair_rates(sp, sd, torch, ct, dev, scan=args.full)
    also.update({k: rr[k] for k in ("repaired_candidates_per_s_perturbed", "repaired_candidates_per_s_uniform")})
    br = batched_runs(torch, ct, W, dev)
    also.update({k: br[k] for k in ("batched_runs_per_s", "batched_runs_per_s_launch_per_generation",
                                  "plain_runs_per_s_same_runs", "batched_vs_plain")})

    sub = None
    if args.full:
        sub = {"valid_configs_per_s": value,
               "cartesian_points_covered_per_s": world * sd.cartesian_size * args.steps / (ms / 1000.0)}
        sub.update(rr)
        sub.update(br)
        sub.update(repair_paper_rates(sp, sd, torch, ct, dev, "large"))
        med_sd = W.medium_space()
        med = ct.Space.from_def(med_sd)
        med.build()
        sub.update(repair_paper_rates(med, med_sd, torch, ct, dev, "medium", n=256))
        del med
        sub.update(plain_runs(torch, ct, W, dev))
        sub.update(one_percent(torch, ct, W, dev))
        sub.update(surrogate_vs_plain(torch, ct, W, dev))
        sub.update(surrogate_large(torch, ct, sp, table, dev))
        sub.update(surrogate_gain_large(torch, ct, W, sp, sd, dev))
        sub.update(aware_vs_unaware(torch, ct, W, dev))
        sub.update(operator_variants(torch, ct, W, dev))
    del table

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": dict(CONFIG, parallelism=f"replicas x{world}"),
           "roofline": roofline, "e2e": e2e, "gpu_launches": launches,
           "clocks": clocks.summary(t0, t1), "also": also}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        if sub is not None:
            blob = json.dumps({"submetrics": sub})
            if args.submetrics_out:
                with open(args.submetrics_out, "w") as f:
                    f.write(blob + "\n")
            print(blob, flush=True)
        print(json.dumps(out), flush=True)   # the headline: always the last line on stdout
    if dist:
        dist.destroy_process_group()
    return 0


def repair_rates(sp, sd, torch, ct, dev, scan=True):
    """Repaired candidates per second on the large space: batches of 256 DE-like perturbations
    of valid keys, and batches of 256 uniform random tuples (worst case); with `scan`, also the
    exhaustive scan alone for 1 to 32 pending candidates."""
    from paper_2606_28372_b300 import workloads as W
    keys = sp.keys()
    res = {}
    for kind in ("perturbed", "uniform"):
        batches = []
        for b in range(8):
            if kind == "uniform":
                t = W.uniform_tuples(sd, 256, seed=100 + b)
            else:
                ranks = torch.from_numpy(W.random_ranks(keys.numel(), 256, seed=200 + b)).to(dev)
                base = sp.unpack(keys[ranks].cpu().numpy().view(np.uint64))
                t = W.perturbed_tuples(sd, base, seed=300 + b)
            batches.append(torch.from_numpy(sp.pack(t).view(np.int64)).to(dev))
        out = torch.empty(256, dtype=torch.int64, device=dev)
        dist = torch.empty(256, dtype=torch.uint8, device=dev)
        for c in batches[:2]:
            sp.repair(c, out, dist)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 4
        e0.record()
        ds = []
        for _ in range(reps):
            for c in batches:
                sp.repair(c, out, dist)
        e1.record()
        torch.cuda.synchronize()
        for c in batches:
            sp.repair(c, out, dist)
            ds.append(dist.cpu().numpy())
        ms = e0.elapsed_time(e1)
        d = np.concatenate(ds)
        res[f"repaired_candidates_per_s_{kind}"] = reps * len(batches) * 256 / (ms / 1000.0)
        res[f"repair_distance_hist_{kind}"] = np.bincount(d, minlength=8)[:8].tolist()
    if not scan:
        return res
    # exhaustive scan alone (scan-only mode): one pass over the 5.56 GB of keys per call
    unif = torch.from_numpy(sp.pack(W.uniform_tuples(sd, 64, seed=999)).view(np.int64)).to(dev)
    sp.set_repair_mode(1, 0)
    scan = {}
    for q in (1, 2, 4, 8, 32):
        c = unif[:q].contiguous()
        o = torch.empty(q, dtype=torch.int64, device=dev)
        sp.repair(c, o)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            sp.repair(c, o)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        scan[f"q{q}"] = {"ms_per_pass": ms, "key_stream_GBps": 8 * keys.numel() / (ms / 1000.0) / 1e9}
    sp.set_repair_mode(0, 0)
    hbm, _ = peaks()
    for q, v in scan.items():
        v["pairs_per_s"] = keys.numel() * int(q[1:]) / (v["ms_per_pass"] / 1000.0)
        v["key_stream_frac_of_copy_peak"] = v["key_stream_GBps"] / hbm
    res["scan_only_repair"] = scan
    return res


def repair_paper_rates(sp, sd, torch, ct, dev, label, n=64, reps=3):
    """The paper's repair rules (index distance, Algorithm 2, Algorithm 3) on `n` DE-like
    perturbations of valid keys: candidates/s, and the streaming pass's rate in
    (valid key, pending candidate) pairs/s and key bytes/s (one pass per 8 pending)."""
    from paper_2606_28372_b300 import workloads as W
    keys = sp.keys()
    nv = keys.numel()
    ranks = torch.from_numpy(W.random_ranks(nv, n, seed=41)).to(dev)
    base = sp.unpack(keys[ranks].cpu().numpy().view(np.uint64))
    tup = W.perturbed_tuples(sd, base, seed=42)
    cand = torch.from_numpy(sp.pack(tup).view(np.int64)).to(dev)
    rk = torch.empty(n, dtype=torch.int64, device=dev)
    sp.lookup(cand, rk)
    pending = int((rk < 0).sum())
    r = np.array(sd.n_values)
    eps = float(np.float32(1.0 / (r.max() - 1)))
    pos = torch.from_numpy((tup * eps).astype(np.float32).ravel()).to(dev)
    words = torch.from_numpy((np.arange(n, dtype=np.int64) * 2654435761 % (1 << 31)).astype(np.int32)).to(dev)
    out = torch.empty(n, dtype=torch.int64, device=dev)
    res = {"pending": pending, "candidates": n, "n_valid": nv}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rule in (1, 2, 3):
        sp.repair_paper(rule, cand, out, pos=pos, eps=eps, words=words)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            sp.repair_paper(rule, cand, out, pos=pos, eps=eps, words=words)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / reps / 1000.0
        res[f"rule{rule}"] = {"ms_per_call": 1000 * sec, "candidates_per_s": n / sec,
                              "pairs_per_s": nv * pending / sec,
                              "key_stream_GBps": 8 * nv * ((pending + 7) // 8) / sec / 1e9}
    return {f"repair_paper_{label}": res}


def plain_runs(torch, ct, W, dev, gens=500, chunk=50):
    """Plain single-run form on the medium space: one run per optimizer, pop 128, 500 generations,
    replayed as CUDA graphs of 50 generations; also unique evaluations to reach 1% of the optimum."""
    sd = W.medium_space()
    sp = ct.Space.from_def(sd)
    sp.build()
    keys = sp.keys().cpu().numpy().view(np.uint64)
    table = W.smooth_table(sd, sp.unpack(keys), seed=0)
    dt = torch.from_numpy(table).to(dev)
    sp.set_fitness(dt)
    tgt = float(np.float32(1.01 * float(table.min())))
    res, total = {}, 0.0
    for kind in ("de", "pso", "firefly", "ga"):
        torch.cuda.synchronize()
        host_warm()
        t0 = time.perf_counter()
        o = ct.Opt(sp, kind, 128, seed=0, target=tgt)
        o.run_graph(0, 1)
        for g in range(1, gens + 1, chunk):
            o.run_graph(g, chunk)
        b = o.best()
        dt_s = time.perf_counter() - t0
        total += dt_s
        res[f"plain_run_ms_{kind}"] = 1000 * dt_s
        res[f"evals_to_1pct_{kind}"] = b["hit_evals"]
        del o
    res["plain_runs_per_s_medium"] = 4 / total
    return res


def batched_runs(torch, ct, W, dev, n_runs=4096, gens=100, plain_sample=48):
    """Batched form: 4096 runs over the 32 batched spaces (mixed DE/PSO/GA, pop 32..128, seed r),
    `gens` generations as one CUDA graph of persistent launches, launch shape autotuned; against
    the same run definitions done one at a time through the single-run path (a sample of them)."""
    import tempfile
    spaces, mins = [], []
    for si in range(32):
        sd = W.batched_space(si)
        sp = ct.Space.from_def(sd)
        sp.build()
        keys = sp.keys().cpu().numpy().view(np.uint64)
        table = torch.from_numpy(W.smooth_table(sd, sp.unpack(keys), seed=si)).to(dev)
        sp.set_fitness(table)
        sp._table_ref = table
        spaces.append(sp)
        mins.append(float(table.min()))
    kinds = ["de", "pso", "ga"]
    runs = [(r % 32, kinds[r % 3], 32 * (1 + (r // 3) % 4), r, float(np.float32(1.01 * mins[r % 32])))
            for r in range(n_runs)]
    b = ct.Batch(spaces, runs)
    cache = os.path.join(tempfile.gettempdir(), "catune_batch_autotune.jsonl")
    th, cps, tune_ms = b.autotune(cache, gens=3)
    b.run_graph(gens)                                  # capture + first replay (warm-up)
    torch.cuda.synchronize()
    b.reset()
    l0 = ct.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.run_graph(gens)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    batched_launches = ct.launch_count() - l0
    res = b.results()
    # the same runs with one persistent launch per generation (a graph of `gens` kernel nodes)
    b.set_gens_per_launch(1)
    b.reset()
    b.run_graph(gens)                                  # capture + first replay (warm-up)
    torch.cuda.synchronize()
    b.reset()
    e0.record()
    b.run_graph(gens)
    e1.record()
    torch.cuda.synchronize()
    ms_per_gen_launch = e0.elapsed_time(e1)
    same_per_gen = bool(np.array_equal(b.results()["best_key"], res["best_key"]))
    b.set_gens_per_launch(0)
    hits = res["hit_evals"][res["hit_evals"] >= 0]
    # the same runs, one at a time (plain path: per-generation kernels, graph replay per run)
    torch.cuda.synchronize()
    host_warm()
    t0 = time.perf_counter()
    plain_hits = []
    for r in range(plain_sample):
        si, kind, pop, seed, tgt = runs[r]
        o = ct.Opt(spaces[si], kind, pop, seed, target=tgt)
        o.run_graph(0, 1)
        o.run_graph(1, gens - 1)
        plain_hits.append(o)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    plain_hits = [o.best()["hit_evals"] for o in plain_hits]   # read after the timed region
    del b
    batched = n_runs / (ms / 1000.0)
    plain = plain_sample / plain_s
    same = res["hit_evals"][:plain_sample]

    def med(h):
        h = np.asarray(h, dtype=np.float64)
        h = np.where(h >= 0, h, np.inf)
        m = float(np.median(h))
        return m if np.isfinite(m) else None
    return {"batched_runs_per_s": batched, "batched_ms_for_all_runs": ms, "batched_generations": gens,
            "batched_runs_per_s_launch_per_generation": n_runs / (ms_per_gen_launch / 1000.0),
            "batched_launch_per_generation_same_results": same_per_gen,
            "evals_to_1pct_same_runs": {"runs": plain_sample, "plain_median": med(plain_hits),
                                        "batched_median": med(same),
                                        "identical": bool(np.array_equal(np.asarray(plain_hits), np.asarray(same))),
                                        "reached": f"{int((np.asarray(same) >= 0).sum())}/{plain_sample}"},
            "batched_runs": n_runs, "batched_launch": {"threads": th, "ctas_per_sm": cps},
            "batched_kernel_launches": batched_launches,
            "plain_runs_per_s_same_runs": plain, "plain_sample_runs": plain_sample,
            "batched_vs_plain": batched / plain,
            "batched_runs_within_1pct": int(len(hits)),
            "batched_median_evals_to_1pct": float(np.median(hits)) if len(hits) else None}


def operator_variants(torch, ct, W, dev, seeds=16, gens=1500, overhead_us=1000.0):
    """Every DE mutation x crossover and every GA crossover (constraint-aware, Table IV
    populations), `seeds` runs on each of three spaces (density ladder 1.5 % and 6.9 %, tiny),
    each setting one batch: batched runs/s and the mean Eq. 2 score over the three spaces."""
    from paper_2606_28372_b300 import score as PS
    defs = [W.density_space(0), W.density_space(4), W.tiny_space()]
    spaces, base = [], []
    for j, sd in enumerate(defs):
        sp = ct.Space.from_def(sd)
        nv = sp.build()
        keys = sp.keys().cpu().numpy().view(np.uint64)
        t = W.lognormal_table(nv, seed=0) if sd.name == "tiny" else W.smooth_table(sd, sp.unpack(keys), seed=j)
        c = W.eval_cost_table(t, seed=j)
        sp._t = torch.from_numpy(t).to(dev)
        sp._c = torch.from_numpy(c.view(np.int32)).to(dev)
        sp.set_fitness(sp._t)
        sp.set_eval_cost(sp._c)
        spaces.append(sp)
        base.append(PS.Baseline(t, c, overhead_us))
    settings = [("de", dict(de_mutation=m, de_crossover=x)) for m in ct.DE_MUTATIONS for x in ct.DE_CROSSOVERS]
    settings += [("ga", dict(ga_crossover=x)) for x in ct.GA_CROSSOVERS]
    out = {}
    for kind, kw in settings:
        P = PAPER_POP[kind]
        runs = [(j, kind, P, 104729 * s + j, -np.inf) for j in range(len(defs)) for s in range(seeds)]
        b = ct.Batch(spaces, runs, **kw)
        b.set_trace(gens, events=4096)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run_graph(gens)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ev = b.events()
        del b
        sc = [float(PS.run_scores(base[j], [ev[r] for r, run in enumerate(runs) if run[0] == j], pop=P,
                                  overhead_us=overhead_us)["per_run"].mean()) for j in range(len(defs))]
        name = kind + "_" + "_".join(str(v) for v in kw.values())
        out[name] = {"score_eq2": float(np.mean(sc)), "score_by_space": dict(zip([d.name for d in defs], sc)),
                     "runs_per_s": len(runs) / (ms / 1000.0), "batched_ms": ms}
    return {"operator_variants": {"generations": gens, "seeds": seeds, "settings": out}}


def run_aware(args):
    import torch
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    print(json.dumps(aware_vs_unaware(torch, ct, W, torch.device("cuda", 0))))
    return 0


def run_batched(args):
    import torch
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    print(json.dumps(batched_runs(torch, ct, W, torch.device("cuda", 0))))
    return 0


def run_surrogate_step(args):
    """Milliseconds per generation of DE at pop 256 on the large space: plain, and forced to screen
    a pool of 16 x 256 candidates every generation (--steps generations after generation 0)."""
    import torch
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    dev = torch.device("cuda", 0)
    sd = W.SPACES[args.workload]()
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    table = torch.exp(torch.randn(nv, generator=g, device=dev, dtype=torch.float32))
    sp.set_fitness(table)
    out = surrogate_large(torch, ct, sp, table, dev, gens=args.steps)
    # fixed-order fp32 work of a screened generation (CUDA cores, two operations per fused
    # multiply-add): forward passes of the 16 x P pool and of the P evaluated configurations, then
    # 8 training steps of 256 (forward and backward)
    N, H, P, pool, steps, bt = len(sd.params), 256, POP, 16, 8, 256
    fwd = H * N + H + 2 * (2 * H * H + H) + 2 * H + 1
    bwd = H + 2 * (2 * H * H) + 2 * (2 * H * H) + 2 * H + (3 * H + 1) + N * H
    flop = (pool * P + P) * fwd + steps * bt * (fwd + bwd)
    peak = ct.measure_fp32_peak()
    ms = out["surrogate_large_de_pop256"]["forced"]["ms_per_generation"]
    out["forced_fp32_flop_per_generation"] = flop
    out["forced_fp32_tflops"] = flop / (ms / 1000.0) / 1e12
    out["fp32_peak_tflops_measured"] = peak / 1e12
    out["forced_frac_of_fp32_peak"] = flop / (ms / 1000.0) / peak
    print(json.dumps({"mode": "surrogate_step", "workload": args.workload, **out}))
    return 0


def run_surrogate(args):
    import torch
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    dev = torch.device("cuda", 0)
    sd = W.large_space()
    sp = ct.Space.from_def(sd)
    sp.build()
    print(json.dumps(surrogate_gain_large(torch, ct, W, sp, sd, dev)))
    return 0


def run_rules(args):
    import torch
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    sd = W.SPACES[args.workload]()
    sp = ct.Space.from_def(sd)
    sp.build()
    print(json.dumps(repair_paper_rates(sp, sd, torch, ct, torch.device("cuda", 0), args.workload)))
    return 0


def run_variants(args):
    import torch
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    print(json.dumps(operator_variants(torch, ct, W, torch.device("cuda", 0))))
    return 0


def run_scan(args):
    """Exhaustive repair scan alone: scan-only repair of 1 to 32 uniform candidates per call,
    one pass over the valid keys each (timed with CUDA events on the launching stream)."""
    import torch
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    dev = torch.device("cuda", 0)
    sd = W.SPACES[args.workload]()
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    sp.set_repair_mode(1, 0)
    unif = torch.from_numpy(sp.pack(W.uniform_tuples(sd, 32, seed=999)).view(np.int64)).to(dev)
    hbm, kind = peaks()
    res = {}
    for q in (1, 2, 4, 8, 16, 32):
        c = unif[:q].contiguous()
        o = torch.empty(q, dtype=torch.int64, device=dev)
        for _ in range(args.warmup):
            sp.repair(c, o)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            sp.repair(c, o)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        gbs = 8 * nv / (ms / 1000.0) / 1e9
        res[f"q{q}"] = {"ms_per_call": ms, "key_stream_GBps": gbs, "frac_of_copy_peak": gbs / hbm,
                        "pairs_per_s": nv * q / (ms / 1000.0)}
    smem = ct.measure_smem_peak()
    print(json.dumps({"mode": "scan", "workload": args.workload, "n_valid": nv, "peak_GBps": hbm,
                      "peak_kind": kind, "smem_wavefront_peak_per_s": smem,
                      "smem_peak_kind": "measured: ct_measure_smem_peak (16-byte shared loads, every SM)",
                      "results": res}))
    return 0


def run_generation(args):
    """One single-run generation at pop 256 on --workload, per optimizer: generations 0 to 4
    untimed (the step graph is captured after the first eager steps), then --steps generations
    timed with CUDA events on the launching stream."""
    import torch
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    dev = torch.device("cuda", 0)
    sd = W.SPACES[args.workload]()
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    table = torch.exp(torch.randn(nv, generator=g, device=dev, dtype=torch.float32))
    sp.set_fitness(table)
    res = {}
    for kind in ("de", "pso", "ga"):
        o = ct.Opt(sp, kind, POP, 7)
        for gen in range(5):
            o.step(gen)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for gen in range(5, 5 + args.steps):
            o.step(gen)
        e1.record()
        torch.cuda.synchronize()
        res[kind] = {"ms_per_generation": e0.elapsed_time(e1) / max(1, args.steps)}
        del o
    print(json.dumps({"mode": "generation", "workload": args.workload, "pop": POP, "steps": args.steps,
                      "results": res}))
    return 0


def run_repair(args):
    """Repair alone on --workload: calls of 256 uniform random tuples and 256 DE-like perturbations
    of valid keys, per radius cap of the ball search (--radius; the cost-model radius by default),
    milliseconds per call (CUDA events on the launching stream)."""
    import torch
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    dev = torch.device("cuda", 0)
    sd = W.SPACES[args.workload]()
    sp = ct.Space.from_def(sd)
    nv = sp.build()
    keys = sp.keys()
    kinds = [args.kind] if args.kind != "both" else ["perturbed", "uniform"]
    res = {}
    for kind in kinds:
        if kind == "uniform":
            t = W.uniform_tuples(sd, 256, seed=100)
        else:
            ranks = torch.from_numpy(W.random_ranks(nv, 256, seed=200)).to(dev)
            t = W.perturbed_tuples(sd, sp.unpack(keys[ranks].cpu().numpy().view(np.uint64)), seed=300)
        c = torch.from_numpy(sp.pack(t).view(np.int64)).to(dev)
        out = torch.empty(256, dtype=torch.int64, device=dev)
        dist = torch.empty(256, dtype=torch.uint8, device=dev)
        res[kind] = {}
        for r in (args.radius or [0]):
            sp.set_repair_mode(2 if r else 0, r)
            for _ in range(args.warmup):
                sp.repair(c, out, dist)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                sp.repair(c, out, dist)
            e1.record()
            torch.cuda.synchronize()
            res[kind][f"radius_{r}" if r else "auto"] = {
                "ms_per_call": e0.elapsed_time(e1) / max(1, args.steps),
                "distance_hist": np.bincount(dist.cpu().numpy(), minlength=8)[:8].tolist()}
        sp.set_repair_mode(0, 0)
    print(json.dumps({"mode": "repair", "workload": args.workload, "n_valid": nv, "results": res}))
    return 0


def surrogate_large(torch, ct, sp, table, dev, gens=10):
    """The surrogate at the large size: DE pop 256 on the large space, milliseconds per
    generation for the plain run, for a run whose judge decides (the lognormal table holds
    nothing to learn, so it mostly stays off), and for one forced to screen every generation
    (a pool of 16 x 256 = 4,096 repaired candidates, all predicted, plus 8 training steps)."""
    logt = torch.log(table)
    out = {}
    for mode in ("plain", "judged", "forced"):
        o = ct.Opt(sp, "de", POP, seed=11)
        if mode == "judged":
            o.set_surrogate(logt)
        elif mode == "forced":
            o.set_surrogate(logt, warmup_mult=0, mae_ratio=1e30)
        o.step(0)
        torch.cuda.synchronize()
        host_warm()
        screened = 0
        t0 = time.perf_counter()
        for g in range(1, gens + 1):
            o.step(g)
            if mode != "plain":
                screened += o.surrogate_info()["screened"]
        torch.cuda.synchronize()
        out[mode] = {"ms_per_generation": 1000 * (time.perf_counter() - t0) / gens, "screened_generations": screened}
        del o
    return {"surrogate_large_de_pop256": out}


def surrogate_gain_large(torch, ct, W, sp, sd, dev, seeds=8, gens=300, chunk=1 << 25):
    """Surrogate against the plain optimizer on the large space with a learnable table: the smooth
    bowl of the medium workload over all 695M valid configurations, built on the device from
    their value indices (ct_unpack_keys_device, 32M keys at a time).  DE and GA at pop 256, 16x
    pool, `seeds` seeds, `gens` generations: median unique evaluations to come within 2 / 5 / 10 %
    of the table's optimum, and the best after 2,000 unique evaluations."""
    keys = sp.keys()
    nv = keys.numel()
    n = len(sd.params)
    table = torch.empty(nv, dtype=torch.float32, device=dev)
    idx = torch.empty(min(chunk, nv) * n, dtype=torch.int32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20240)
    for s0 in range(0, nv, chunk):
        k = keys[s0:s0 + chunk]
        part = idx[: k.numel() * n].view(k.numel(), n)
        sp.unpack_device(k, part)
        table[s0:s0 + k.numel()] = W.smooth_table_device(sd, part, seed=0, generator=gen)
    del idx
    sp.set_fitness(table)
    logt = torch.log(table)
    opt = float(table.min())
    out = {}
    for kind in ("de", "ga"):
        for mode in ("plain", "surrogate"):
            curves = []
            for seed in range(seeds):
                o = ct.Opt(sp, kind, POP, seed)
                if mode == "surrogate":
                    o.set_surrogate(logt)
                cu = []
                for g in range(gens + 1):
                    o.step(g)
                    b = o.best()
                    cu.append((b["n_unique"], b["best_fit"] / opt))
                curves.append(cu)
                del o
            rec = {}
            for pct in (2, 5, 10):
                first = [next((m for m, f in cu if f <= 1 + pct / 100), None) for cu in curves]
                hit = [x for x in first if x is not None]
                rec[f"evals_to_{pct}pct_median"] = float(np.median(hit)) if len(hit) * 2 > len(first) else None
                rec[f"reached_{pct}pct"] = f"{len(hit)}/{len(first)}"
            rec["best_rel_after_2000_evals"] = float(np.median([[f for m, f in cu if m <= 2000][-1] for cu in curves]))
            out[f"surrogate_large_{kind}_{mode}"] = rec
    return out


def surrogate_vs_plain(torch, ct, W, dev, seeds=16, gens=150):
    """Unique evaluations to come within 1/2/5 % of the table optimum, and the best fitness after
    1000 unique evaluations (medians over seeds), for plain and surrogate-screened DE and GA on
    the medium space at pop 128."""
    sd = W.medium_space()
    sp = ct.Space.from_def(sd)
    sp.build()
    keys = sp.keys().cpu().numpy().view(np.uint64)
    table = W.smooth_table(sd, sp.unpack(keys), seed=0)
    dt = torch.from_numpy(table).to(dev)
    sp.set_fitness(dt)
    logt = torch.from_numpy(np.log(table.astype(np.float64)).astype(np.float32)).to(dev)
    opt = float(table.min())
    out = {}
    for kind in ("de", "ga"):
        for mode in ("plain", "surrogate"):
            curves = []
            for seed in range(seeds):
                o = ct.Opt(sp, kind, 128, seed)
                if mode == "surrogate":
                    o.set_surrogate(logt)
                cu = []
                for g in range(gens + 1):
                    o.step(g)
                    b = o.best()
                    cu.append((b["n_unique"], b["best_fit"] / opt))
                curves.append(cu)
            rec = {}
            for pct in (1, 2, 5):
                first = [next((n for n, f in cu if f <= 1 + pct / 100), None) for cu in curves]
                hit = [x for x in first if x is not None]
                rec[f"evals_to_{pct}pct_median"] = float(np.median(hit)) if len(hit) * 2 > len(first) else None
                rec[f"reached_{pct}pct"] = f"{len(hit)}/{len(first)}"
            rec["best_rel_after_1000_evals"] = float(np.median([[f for n, f in cu if n <= 1000][-1] for cu in curves]))
            out[f"surrogate_cmp_{kind}_{mode}"] = rec
    return out


def _median_hits(h):
    """Median unique evaluations to the target over all runs (a run that never got there counts as
    infinitely many); None when fewer than half got there."""
    h = np.asarray(h, dtype=np.float64)
    m = float(np.median(np.where(h >= 0, h, np.inf)))
    return m if np.isfinite(m) else None


def one_percent(torch, ct, W, dev, seeds=16):
    """The 1 % criterion.  (1) Census of the smooth tables: how many configurations lie within
    1 / 2 / 5 % of each table's optimum, and the second best's ratio to it.  (2) Plain against
    surrogate-screened DE and GA: unique evaluations until the best is within 1 % of the optimum
    (medians over `seeds` seeds, runs that never get there counted as infinitely many), on a batched
    space of 22,386 valid configurations (pop 64, 200 generations) and on the medium space
    (pop 128, 600 generations)."""
    census, out = {}, {}
    cases = [("medium", W.medium_space(), 0, 128, 600), ("batched_5", W.batched_space(5), 5, 64, 200),
             ("batched_10", W.batched_space(10), 10, 64, 200)]
    for name, sd, tseed, pop, gens in cases:
        sp = ct.Space.from_def(sd)
        sp.build()
        keys = sp.keys().cpu().numpy().view(np.uint64)
        t = W.smooth_table(sd, sp.unpack(keys), seed=tseed)
        srt = np.sort(t)
        census[name] = {"valid": int(len(t)), "second_best_rel": float(srt[1] / srt[0]),
                        **{f"within_{p}pct": int((t <= np.float32((1 + p / 100) * srt[0])).sum()) for p in (1, 2, 5)}}
        if name == "batched_10":
            continue
        dt = torch.from_numpy(t).to(dev)
        sp.set_fitness(dt)
        logt = torch.from_numpy(np.log(t.astype(np.float64)).astype(np.float32)).to(dev)
        tgt = float(np.float32(1.01 * float(srt[0])))
        for kind in ("de", "ga"):
            for mode in ("plain", "surrogate"):
                hits = []
                for seed in range(seeds):
                    o = ct.Opt(sp, kind, pop, seed, target=tgt)
                    if mode == "surrogate":
                        o.set_surrogate(logt)
                    for g in range(gens + 1):
                        o.step(g)
                    hits.append(o.best()["hit_evals"])
                    del o
                reached = [h for h in hits if h >= 0]
                out[f"{name}_{kind}_{mode}"] = {
                    "evals_to_1pct_median": _median_hits(hits),
                    "evals_to_1pct_median_of_reached": float(np.median(reached)) if reached else None,
                    "reached": f"{len(reached)}/{seeds}", "pop": pop, "generations": gens}
    return {"one_percent": {"census": census, "runs": out}}


def run_one_percent(args):
    import torch
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    from paper_2606_28372_b300 import workloads as W
    print(json.dumps(one_percent(torch, ct, W, torch.device("cuda", 0))))
    return 0


PAPER_POP = {"de": 160, "pso": 30, "firefly": 20, "ga": 20}   # Table IV (DE: 16 x 10 parameters)


def aware_vs_unaware(torch, ct, W, dev, seeds=16, overhead_us=1000.0, K=50, gens=(4000, 24000)):
    """Synthetic analogue of the aware-vs-default comparison of Section V-B, scored by Eq. 2.

    The four optimizers with Table IV's population sizes, constraint-aware and not (random
    Cartesian start, no repair, static penalty), `seeds` runs each on the eight spaces of the
    density ladder (1.5 % .. 100 %) and the tiny space (56 %); every run of one mode advances in
    one batched launch per generation and logs every improvement of its best with the simulated
    clock at that evaluation (proposals evaluated one at a time; each configuration's synthetic
    compile + 7 runs charged once, plus `overhead_us` per proposal).  Each run is scored against the space's random-search baseline over the budget of
    Section V-A.  Aware runs get gens[0] generations, the cheaper non-aware ones gens[1]; a run
    whose clock ends before the budget keeps its last value ("truncated")."""
    from scipy.stats import spearmanr
    from paper_2606_28372_b300 import score as PS
    kinds = ["de", "pso", "firefly", "ga"]
    defs = [W.density_space(j) for j in range(8)] + [W.tiny_space()]
    spaces, dens, opt, base = [], [], [], []
    for j, sd in enumerate(defs):
        sp = ct.Space.from_def(sd)
        nv = sp.build()
        keys = sp.keys().cpu().numpy().view(np.uint64)
        t = W.lognormal_table(nv, seed=0) if sd.name == "tiny" else W.smooth_table(sd, sp.unpack(keys), seed=j)
        c = W.eval_cost_table(t, seed=j)
        sp._table_ref = torch.from_numpy(t).to(dev)
        sp._cost_ref = torch.from_numpy(c.view(np.int32)).to(dev)
        sp.set_fitness(sp._table_ref)
        sp.set_eval_cost(sp._cost_ref)
        spaces.append(sp)
        dens.append(nv / sd.cartesian_size)
        opt.append(float(t.min()))
        base.append(PS.Baseline(t, c, overhead_us))
    S = len(defs)
    runs = [(j, k, PAPER_POP[k], 7919 * s + 31 * j + ki, float(np.float32(1.01 * opt[j])))
            for j in range(S) for ki, k in enumerate(kinds) for s in range(seeds)]
    budgets = [b.budget() for b in base]
    table, ms, score = {}, {}, {}
    for mode, aware, G in (("aware", 1, gens[0]), ("unaware", 0, gens[1])):
        b = ct.Batch(spaces, runs, constraint_aware=aware)
        b.set_trace(G, events=4096)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(G // 1000):
            b.run_graph(1000)
        e1.record()
        torch.cuda.synchronize()
        ms[mode] = e0.elapsed_time(e1)
        tr = b.trace()
        ev = b.events()
        del b
        for j in range(S):
            for ki, k in enumerate(kinds):
                rows = [r for r, run in enumerate(runs) if run[0] == j and run[1] == k]
                P = PAPER_POP[k]
                res = PS.run_scores(base[j], [ev[r] for r in rows], pop=P, overhead_us=overhead_us, K=K)
                clock_end = tr["cost"][rows, -1].astype(np.float64) + G * P * overhead_us
                B = budgets[j][1]
                clock = tr["cost"][rows].astype(np.float64) + np.arange(1, G + 1) * P * overhead_us
                hit = (tr["best_fit"][rows] <= np.float32(1.01 * opt[j])) & (clock <= B)
                score[(j, k, mode)] = float(res["per_run"].mean())
                table.setdefault(f"{defs[j].name}_{100 * dens[j]:.2f}pct_{k}", {})[mode] = {
                    "score": score[(j, k, mode)],
                    "score_sem": float(res["per_run"].std(ddof=1) / np.sqrt(len(rows))),
                    "within_1pct_in_budget": float(hit.any(axis=1).mean()),
                    "truncated": float((clock_end < B).mean())}
    agg = {m: {k: float(np.mean([score[(j, k, m)] for j in range(S)])) for k in kinds} for m in ("aware", "unaware")}
    gain = {k: [score[(j, k, "aware")] - score[(j, k, "unaware")] for j in range(S)] for k in kinds}
    corr = {k: float(spearmanr(dens, gain[k]).statistic) for k in kinds}
    return {"aware_vs_unaware": {
        "score_eq2_by_kind": agg,
        "score_gain_by_kind": {k: agg["aware"][k] - agg["unaware"][k] for k in kinds},
        "score_gain_mean": float(np.mean([agg["aware"][k] - agg["unaware"][k] for k in kinds])),
        "spearman_density_vs_gain": corr, "per_space": table,
        "budget_s": {defs[j].name: budgets[j][1] / 1e6 for j in range(S)},
        "budget_draws": {defs[j].name: budgets[j][0] for j in range(S)},
        "generations": {"aware": gens[0], "unaware": gens[1]}, "seeds": seeds, "pop": PAPER_POP,
        "overhead_ms_per_proposal": overhead_us / 1000, "time_points": K,
        "batched_ms": ms, "runs_per_mode": len(runs)}}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--quick", action="store_true", help="headline step only (no rebuild, e2e, other parts or CPU leg)")
    ap.add_argument("--full", action="store_true",
                    help="also every sub-metric (repair rules, plain runs, surrogate, aware vs unaware, operator "
                         "variants; minutes), printed as one JSON line before the headline")
    ap.add_argument("--submetrics-out", default=None, help="with --full: also write the sub-metrics line to this file")
    ap.add_argument("--host-warm", type=float, default=HOST_WARM_S,
                    help="seconds of continuous host work before each timed region (0 for profiler runs, whose "
                         "numbers are never bench values)")
    ap.add_argument("--mode", default="step",
                    choices=["step", "scan", "repair", "aware", "variants", "batched", "rules", "surrogate",
                             "surrogate_step", "onepct", "generation"],
                    help="scan: only the exhaustive repair scan (scan-only repair of 1 to 32 uniform candidates); "
                         "repair: only repair calls of 256 candidates on --workload (--kind, --radius); "
                         "aware: only the constraint-aware vs non-aware comparison over the density ladder; "
                         "variants: only the DE/GA operator comparison; batched: only the batched-runs "
                         "comparison; rules: only the paper's repair rules on --workload; surrogate: only the "
                         "surrogate-vs-plain comparison on the large space; surrogate_step: milliseconds per "
                         "generation of plain, judged and forced-screening DE on --workload; onepct: the 1 %% "
                         "criterion (table census, plain against surrogate-screened runs); generation: device "
                         "milliseconds per single-run generation of DE, PSO and GA at pop 256 on --workload")
    ap.add_argument("--workload", default="large", choices=["large", "large_slice"],
                    help="large_slice: the same kernels on a 146M-key slice, for hardware-counter captures")
    ap.add_argument("--kind", default="both", choices=["both", "perturbed", "uniform"],
                    help="repair mode: the candidates")
    ap.add_argument("--radius", type=int, nargs="*", default=None,
                    help="repair mode: ball radius caps to time (default: the cost-model radius)")
    a = ap.parse_args()
    HOST_WARM_S = a.host_warm
    if a.impl == "reference":
        sys.exit(run_reference(a))
    if a.mode == "aware":
        sys.exit(run_aware(a))
    if a.mode == "variants":
        sys.exit(run_variants(a))
    if a.mode == "batched":
        sys.exit(run_batched(a))
    if a.mode == "surrogate":
        sys.exit(run_surrogate(a))
    if a.mode == "surrogate_step":
        sys.exit(run_surrogate_step(a))
    if a.mode == "onepct":
        sys.exit(run_one_percent(a))
    if a.mode == "rules":
        sys.exit(run_rules(a))
    if a.mode == "repair":
        sys.exit(run_repair(a))
    if a.mode == "generation":
        sys.exit(run_generation(a))
    sys.exit(run_scan(a) if a.mode == "scan" else run_ours(a))
