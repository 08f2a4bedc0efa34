"""Benchmark of the signed-particle Wigner Monte Carlo hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload NAME]

A step is one pass of the whole hot path over the ensemble: survivor
enumeration and occupied cells (rule 2 rebuild), the Wigner kernel on the
occupied cells with gamma and the momentum CDF, and the particle step (drift,
absorption, pair creation, signed histogram).  The default workload is the
16384-cell noisy double barrier (Q = n_M = 1024) with 1e8 particles, where
every occupied cell creates pairs; the 2000-cell barrier (1e7 particles, whose
early steps create no pairs) is a secondary drift-only leg.  `value` is particle-steps/s
over all ranks; N > 1 runs independent replicas (one simulation per rank, its
own Philox stream), so scaling is weak.  `--impl reference` times the CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import wmc_inputs as wi  # noqa: E402

METRIC = "particle-steps/s; kernel cell·M evals/s at stated err vs FP64 (TC vs FP32)"
UNIT = "particle-steps/s"
L2_BYTES = 129 * 2 ** 20

# DRAM bytes (read + write) of one particle-step kernel launch from the ncu
# capture named below; None until the current kernel has been captured.
K_STEP_DRAM_BYTES = 23258368
K_STEP_TRAFFIC_SOURCE = ("ncu --set full capture of k_step on double-barrier-16384 (5th launch): dram read "
                         "23.26 MB + write 0 per launch (profiles/k_step_double-barrier-16384.md)")
# DRAM bytes of one BF16 launch of k_kernel_eval_tc_ta on all 16384 cells (the sine image and the potential
# come from L2 after the first touch; the 32 MB of output rows stay in L2)
TC_TA_DRAM_BYTES = 743424 + 1280
TC_TA_DRAM_SOURCE = ("ncu --set full capture of k_kernel_eval_tc_ta<BF16> on double-barrier-16384 (4th launch): "
                     "dram read 743.4 KB + write 1.3 KB (profiles/k_kernel_eval_tc_ta_double-barrier-16384.md)")


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # live before the work starts: wait (at most 3 s) for the first sample
            t_end = time.time() + 3.0
            while not self.lines and time.time() < t_end:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- CPU oracle leg
def oracle_rate(w, budget_s: float, n_steps_min: int = 1, max_steps: int = 1000):
    """Oracle particle-steps/s on w, stepping until budget_s has elapsed."""
    import oracle
    p = oracle.params(w)
    V = wi.potential(w)
    h = wi.initial_histogram(w)
    ps = 0
    t_used = 0.0
    steps = 0
    t = 1
    while steps < max_steps and (steps < n_steps_min or t_used < budget_s):
        t0 = time.perf_counter()
        h, st = oracle.simulate(p, h, t, 1, V=V)
        t_used += time.perf_counter() - t0
        ps += int(st[oracle.ST_PARTICLE_STEPS])
        steps += 1
        t += 1
    return ps / t_used, ps, steps, t_used


def reference_arm(args, w):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    # size each step's sample so that the whole run stays within about 3 minutes
    per_step_budget = 150.0 / max(1, args.steps + args.warmup)
    rate0, _, _, _ = oracle_rate(wi.scaled(w, 200_000), 0.0)
    n0 = int(min(w.packet.n0, max(20_000, rate0 * per_step_budget)))
    ws = wi.scaled(w, n0)
    oracle_rate(ws, 0.0, n_steps_min=args.warmup, max_steps=args.warmup) if args.warmup else None
    rate, ps, steps, secs = oracle_rate(ws, 0.0, n_steps_min=args.steps, max_steps=args.steps)
    sample = f"{w.name} with N0={n0} (packet shape kept), {steps} oracle steps, {secs:.1f} s"
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_x": w.n_x, "Q": w.Q, "n_M": w.n_M, "N0": n0, "kernel": "fp64 oracle"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- native arm
def reduce_over_ranks(ms, particle_steps, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the
    particle-steps) -- the whole-job time is the slowest replica's.  A single
    process returns its own values."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(ms), float(particle_steps)
    tt = torch.tensor([ms, particle_steps], dtype=torch.float64, device=device)
    mx = tt.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


def native_arm(args, w):
    import torch
    from paper_1806_00082_gb300 import build, wmc

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    wmc.load()

    wl = w.replace(sim=rank)          # independent replica per rank
    p = wmc.Params.of(wl)
    V = torch.from_numpy(wi.potential(wl)).to(dev)
    h0_host = wi.initial_histogram(wl)
    h0 = torch.from_numpy(h0_host).to(dev)
    ws = wmc.workspace(p, dev)
    a = h0.clone()
    b = torch.empty_like(a)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    n_iter = max(1, (args.steps + 1) // 2)      # one timed iteration = one graph launch of 2 steps
    steps = 2 * n_iter
    with torch.cuda.stream(stream):
        wmc.init(p, ws)
        t = 1
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_iter)]
        # clocks sampled from the warm-up steps through the timed region (at 20
        # steps the timed region alone is shorter than one sampling interval)
        clk = Clocks(local).__enter__()
        try:
            for _ in range(max(1, (args.warmup + 1) // 2)):
                wmc.run(p, V, a, b, t, 2, ws)
                t += 2
            wmc.reset_counters(p, ws)
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            for q in range(n_iter):
                flush.zero_()                    # L2 flushed between timed iterations
                ev[q][0].record(stream)
                wmc.run(p, V, a, b, t, 2, ws)
                ev[q][1].record(stream)
                t += 2
            stream.synchronize()
        finally:
            clk.__exit__(None, None, None)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
        c = wmc.get_counters(p, ws)
        err = wmc.get_error(p, ws)
    ms_max, ps_total = reduce_over_ranks(ms, float(c["particle_steps"]), dev)
    value = ps_total / (ms_max * 1e-3)

    # ---- dominant kernel: the particle step inside the same step graphs
    roof = step_roofline(wmc, torch, p, V, a, b, ws, stream, t, flush, min(n_iter, 20), local)
    t += 2 * min(n_iter, 20)
    # ---- end to end through the C ABI with host buffers
    e2e = end_to_end(wmc, torch, p, V, ws, stream, h0_host, a, t + 4, n=12)
    kev = kernel_eval_rate(wmc, torch, dev, stream, flush) if rank == 0 and not args.no_batched else None
    drift = drift_only_rate(wmc, torch, dev, stream, flush) if rank == 0 and not args.no_batched else None
    bat = batched_rate(wmc, torch, dev, stream) if rank == 0 and not args.no_batched else None
    adjo = adjoint_rate(wmc, torch, dev, stream) if rank == 0 and not args.no_batched else None
    n2t = n2_train_rate(wmc, torch, dev, stream) if rank == 0 and not args.no_batched else None

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, ps_cpu, st_cpu, secs = oracle_rate(w, 10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{w.name} full N0={w.packet.n0}, first {st_cpu} step(s) ({secs:.1f} s, single thread; "
                         f"the FP64 kernel on every occupied cell and the particle loop)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_max / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "n_x": w.n_x, "Q": w.Q, "n_M": w.n_M, "N0": w.packet.n0,
                   "dt_fs": w.dt_s / 1e-15,
                   "kernel": ("FP32 accuracy: 3xTF32 tensor cores, per-K-block accumulators" if w.Q > 256
                              else "FP32 (compensated, CUDA cores)"),
                   "parallelism": f"replicas x{world}", "l2": "flushed between timed iterations (2 steps each)"},
        "clocks": clk.summary(),
        # per step: k_rows, k_plan, kernel stage (contraction + CDF, or the fused
        # small-window kernel), k_step, k_pairs; per wmc_run call: k_set_step
        "gpu_launches": (6 if w.Q // 2 > 128 else 5) * steps + n_iter,
        "e2e": e2e,
        "roofline": roof,
        "cpu_baseline": cpu,
        "kernel_eval": kev,
        "drift_only": drift,
        "batched": bat,
        "adjoint": adjo,
        "n2_train": n2t,
        "counters": {k: c[k] for k in ("pairs", "absorbed", "dropped", "n_occ", "population", "flags")},
        "device_status": {"code": err[0], "message": err[1]},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def reach_cells(wmc, torch, p, V, ws, stream):
    """Cells whose particles draw a pair-creation word: gamma > 0 in the cell or
    a neighbour (the potential is static), from the public kernel calls on an
    initialised workspace."""
    occ_all = torch.arange(p.n_x, dtype=torch.int32, device=V.device)
    with torch.cuda.stream(stream):
        VWh = wmc.kernel_eval(p, V, occ_all, ws)
        _, gamma, _ = wmc.kernel_cdf(p, VWh, with_cdf=False)
    stream.synchronize()
    g = gamma > 0
    reach = g.clone()
    reach[1:] |= g[:-1]
    reach[:-1] |= g[1:]
    return reach


def philox_calls(c0, c1, r0, r1):
    """Philox4x32-10 calls of the particle-step kernel per step over one
    two-step launch: one offset draw per four survivors (the particle-step
    counter, exact) and one pair-creation draw per four survivors of reach
    cells (exact for the first step, the launch's output state standing in for
    the second step's input).  The pair draws run in the pair kernel."""
    ps = c1["particle_steps"] - c0["particle_steps"]
    return (ps / 4.0 + (r0 + r1) / 4.0) / 2.0


def philox_peak(wmc, torch, dev, stream, reps=5):
    """Calls per second of the generator alone (wmc_philox_throughput: two
    calls at a time under one key schedule, every SM busy), timed with events;
    the ceiling of the particle step's arithmetic."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.empty(sms * 8 * 256, dtype=torch.int32, device=dev)
    pairs = 128
    best = None
    with torch.cuda.stream(stream):
        wmc.philox_throughput(out, pairs)
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wmc.philox_throughput(out, pairs)
            e1.record(stream)
            stream.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            best = sec if best is None else min(best, sec)
    calls = 2.0 * pairs * out.numel()
    return calls / best, {"threads": out.numel(), "calls_per_launch": calls, "seconds": best, "sms": sms}


# 14 bytes per particle-step: the algorithmic traffic of a stored-particle
# design (7-byte SoA record read and rewritten per step)
BYTES_PER_PARTICLE_STEP = 14


def step_roofline(wmc, torch, p, V, a, b, ws, stream, t, flush, n, gpu_index):
    """The particle-step kernel as it runs in the timed step graphs: n more
    launches of the same two-step graph, L2 flushed before each, recaptured
    with the library's CUDA events around the kernel (event-record nodes on the
    launching stream).  Duration = the second step's kernel of each launch;
    work in Philox4x32-10 calls (philox_calls), against the measured calls/s
    of the generator alone; clocks sampled meanwhile."""
    peaks, src = _peaks()
    reach = reach_cells(wmc, torch, p, V, ws, stream)
    k_ms, k_calls, k_ps = [], [], []
    with Clocks(gpu_index) as clk:
        peak_calls, peak_info = philox_peak(wmc, torch, a.device, stream)
        with torch.cuda.stream(stream):
            wmc.step_timing(True)
            try:
                c0 = wmc.get_counters(p, ws)
                r0 = float(a.abs()[reach].sum())
                for _ in range(n):
                    torch.cuda._sleep(200_000)   # keep the stream busy while the host enqueues after its wait
                    flush.zero_()
                    wmc.run(p, V, a, b, t, 2, ws)
                    t += 2
                    k_ms.append(wmc.step_timing_read())
                    c1 = wmc.get_counters(p, ws)
                    r1 = float(a.abs()[reach].sum())
                    k_calls.append(philox_calls(c0, c1, r0, r1))
                    k_ps.append((c1["particle_steps"] - c0["particle_steps"]) / 2.0)
                    c0, r0 = c1, r1
            finally:
                wmc.step_timing(False)
    sec = float(np.mean(k_ms)) * 1e-3
    per_launch = float(np.mean(k_calls))
    ps_launch = float(np.mean(k_ps))
    achieved = per_launch / sec
    hbm = BYTES_PER_PARTICLE_STEP * ps_launch / sec / 1e9
    return {"bound": "alu", "kernel": "k_step", "achieved": achieved, "peak": peak_calls,
            "unit": "Philox4x32-10 calls/s", "frac": achieved / peak_calls, "traffic": K_STEP_DRAM_BYTES,
            "traffic_source": K_STEP_TRAFFIC_SOURCE,
            "per_launch": {"philox_calls": per_launch, "particle_steps": ps_launch, "seconds": sec,
                           "launches_timed": len(k_ms)},
            "peak_source": "measured in this run: wmc_philox_throughput (the generator alone on every SM, two "
                           f"calls per key schedule), {peak_info['threads']} threads, events; clocks {clk.summary()}",
            "hbm_equivalent": {"bytes_per_particle_step": BYTES_PER_PARTICLE_STEP, "achieved_GBs": hbm,
                               "peak_GBs": peaks["hbm_gbs"], "frac": hbm / peaks["hbm_gbs"],
                               "note": f"{src} copy bandwidth; the design stores no particles, so this is the "
                                       "throughput a stored-particle step would need"}}


def end_to_end(wmc, torch, p, V, ws, stream, h0_host, a_dev, t0, n=12):
    """Per step: H2D of a state from pinned memory, one wmc_run step, D2H of the
    new state, for a sequence of n states (three distinct ones in turn: the
    initial state and two later states of the same run).  The steps run in order
    on the compute stream (they share the workspace); the copies run on their
    own streams into three buffer sets, so that the upload of the next state,
    the download of the previous result and the current step all overlap (with
    two sets an upload would wait for the download of its set's last result).  Timed with
    events from the first upload to the last download (all of it enqueued
    behind a sleep kernel, so that host enqueue time is not timed).  Each
    state and its output (2 x 64 MB at 16384 x 1024) exceed L2 together."""
    states = [torch.from_numpy(h0_host).pin_memory(), a_dev.cpu().pin_memory()]
    with torch.cuda.stream(stream):
        tmp_a, tmp_b = a_dev.clone(), torch.empty_like(a_dev)
        wmc.run(p, V, tmp_a, tmp_b, t0, 2, ws)
        stream.synchronize()
    states.append(tmp_a.cpu().pin_memory())
    del tmp_a, tmp_b
    n_sets = 3
    host_out = [torch.empty_like(states[0]).pin_memory() for _ in range(n_sets)]
    bufs = [(torch.empty_like(a_dev), torch.empty_like(a_dev)) for _ in range(n_sets)]
    up, down = torch.cuda.Stream(device=a_dev.device), torch.cuda.Stream(device=a_dev.device)
    ev = lambda: torch.cuda.Event()
    t0 += 2
    with torch.cuda.stream(stream):
        # warm-up calls: build the cached one-step graphs of both buffer sets
        # outside the timed region
        for a, b in bufs:
            a.copy_(states[0], non_blocking=True)
            wmc.run(p, V, a, b, t0, 1, ws)
        wmc.reset_counters(p, ws)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(4_000_000)
        e0.record(stream)
        free = [None] * n_sets
        done = []
        for q in range(n):
            k = q % n_sets
            a, b = bufs[k]
            up.wait_event(e0)
            if free[k] is not None:
                up.wait_event(free[k])
            with torch.cuda.stream(up):
                a.copy_(states[q % len(states)], non_blocking=True)
                loaded = ev(); loaded.record(up)
            stream.wait_event(loaded)
            wmc.run(p, V, a, b, t0 + q, 1, ws)
            stepped = ev(); stepped.record(stream)
            down.wait_event(stepped)
            with torch.cuda.stream(down):
                host_out[k].copy_(a, non_blocking=True)
                free[k] = ev(); free[k].record(down)
            done.append(free[k])
        for d in done[-n_sets:]:
            stream.wait_event(d)
        e1.record(stream)
        stream.synchronize()
        c = wmc.get_counters(p, ws)
    secs = e0.elapsed_time(e1) * 1e-3
    nbytes = states[0].numel() * 4
    return {"value": c["particle_steps"] / secs, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": n, "states": len(states),
            "overlap": "copies on two streams, three buffer sets"}


def _oracle_rows_worker(args):
    """One process of the oracle kernel timing: FP64 rows of the given cells."""
    import oracle as orc
    wname, rows = args
    w = wi.WORKLOADS[wname]
    V = wi.potential(w)
    t0 = time.perf_counter()
    orc.kernel_rows(orc.params(w.replace(n_M=w.Q)), V, rows)
    return time.perf_counter() - t0


def oracle_kernel_rate(w, rows_single=512, rows_per_proc=256):
    """The FP64 oracle kernel (Eq. wigner-1d-discrete, the direct window sum) in
    cell x M evaluations per second: one thread, then one process per host core
    (spawned) on their own rows."""
    import multiprocessing as mp
    rng = np.random.default_rng(5)
    rows = rng.integers(0, w.n_x, rows_single)
    t1 = _oracle_rows_worker((w.name, rows))
    single = rows_single * w.Q / t1
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_rows_worker, [(w.name, rows[:8])] * cores)   # import and build in every worker
        t0 = time.perf_counter()
        pool.map(_oracle_rows_worker, [(w.name, rng.integers(0, w.n_x, rows_per_proc)) for _ in range(cores)])
        tall = time.perf_counter() - t0
    return {"single_thread": {"cellM_per_s": single, "rows": rows_single, "seconds": t1},
            "all_cores": {"cellM_per_s": cores * rows_per_proc * w.Q / tall, "cores": cores,
                          "rows": cores * rows_per_proc, "seconds": tall},
            "note": "FP64 direct window sum, n_M = Q columns per row (one period)"}


def kernel_eval_rate(wmc, torch, dev, stream, flush, reps=10):
    """The contraction on all 16384 cells of the double barrier (Q = n_M = 1024)
    in each precision form, timed alone with events (L2 flushed before each
    launch).  Algorithmic work: 2 (h-1)^2 flop per cell (distinct columns); the
    split forms issue three products per output (pipe work 3x).  The FP64
    oracle kernel is timed beside it on the host cores."""
    peaks, src = _peaks()
    w = wi.DOUBLE_BARRIER_16384
    p = wmc.Params.of(w)
    V = torch.from_numpy(wi.potential(w)).to(dev)
    ws = wmc.workspace(p, dev)
    occ = torch.arange(w.n_x, dtype=torch.int32, device=dev)
    out = torch.empty((w.n_x, w.Q // 2), dtype=torch.float32, device=dev)
    h = w.Q // 2
    flops = 2.0 * w.n_x * (h - 1) ** 2
    # normwise error bounds asserted by tests/test_gpu_dft.py and tests/test_gpu_tensorcore.py;
    # "fp32" is the FP32-accuracy request (the 3xTF32 tensor-core form at this Q),
    # "fp32_simt" the compensated CUDA-core form
    bounds = {"fp32": 5e-7, "fp32_simt": 5e-7, "bf16": 1.5e-2, "fp16": 1e-3, "fp16_split": 5e-7, "tf32x3": 5e-7}
    res = {}
    with torch.cuda.stream(stream):
        wmc.init(p, ws)
        # FP64 reference rows on the device (sliding window), timed as a form
        ref_rows = torch.empty_like(out)
        wmc.kernel_eval_dft(p, V, ws, out=ref_rows)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wmc.kernel_eval_dft(p, V, ws, out=ref_rows)
        e1.record(stream)
        stream.synchronize()
        dft_sec = e0.elapsed_time(e1) * 1e-3
        ref64 = ref_rows.double()
        scale = float(ref64.abs().max())

        def err_of(rows):
            return float((rows.double() - ref64).abs().max()) / scale

        # about 20 ms of launches first, so that the first form timed does not
        # see the clocks ramping up after the host-side work above
        for _ in range(150):
            wmc.kernel_eval(p, V, occ, ws, prec=wmc.PRECISIONS["fp32"], out=out)
        stream.synchronize()
        for form in ("fp32", "fp32_simt", "bf16", "fp16", "fp16_split", "tf32x3"):
            prec = wmc.PRECISIONS[form]
            for _ in range(3):
                wmc.kernel_eval(p, V, occ, ws, prec=prec, out=out)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                wmc.kernel_eval(p, V, occ, ws, prec=prec, out=out)
                e1.record(stream)
                stream.synchronize()
                tot += e0.elapsed_time(e1) * 1e-3
            sec = tot / reps
            r = {"seconds": sec, "cellM_per_s": w.n_x * w.n_M / sec, "tflops_algorithmic": flops / sec / 1e12,
                 "err_bound_normwise": bounds[form], "err_measured_normwise": err_of(out)}
            if form == "fp32_simt":
                r["bound"] = "fp32 pipe (SIMT)"
            else:
                issued = flops * (3 if form in ("fp16_split", "tf32x3", "fp32") else 1)
                if form in ("tf32x3", "fp32"):  # TF32 pipe: the BF16 peak x the nominal ratio 1.1 / 2.25 PFLOP/s
                    peak = peaks["bf16_tflops"] * 1e12 * (1.1 / 2.25)
                    psrc = f"{src} bf16 dense x 1.1/2.25 (nominal tf32/bf16)"
                else:
                    peak = peaks["bf16_tflops"] * 1e12
                    psrc = f"{src} bf16 dense (fp16 same rate)"
                r["roofline"] = {"bound": "tensor", "achieved": issued / sec / 1e12, "peak": peak / 1e12,
                                 "unit": "TFLOP/s", "frac": issued / sec / peak, "traffic": None,
                                 "peak_source": psrc}
                if form == "bf16":
                    r["roofline"]["traffic"] = TC_TA_DRAM_BYTES
                    r["roofline"]["traffic_source"] = TC_TA_DRAM_SOURCE
            res[form] = r
    # the N = 2 barycentric network (Sec. 2.3) on the same cells
    n2 = {}
    with torch.cuda.stream(stream):
        for form in ("fp32_simt", "bf16", "fp16", "fp16_split"):
            prec = wmc.PRECISIONS[form]
            for _ in range(3):
                wmc.kernel_eval_n2(p, V, occ, ws, prec=prec, out=out)
            tot = 0.0
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                wmc.kernel_eval_n2(p, V, occ, ws, prec=prec, out=out)
                e1.record(stream)
                stream.synchronize()
                tot += e0.elapsed_time(e1) * 1e-3
            sec = tot / reps
            n2[form] = {"seconds": sec, "cellM_per_s": w.n_x * w.n_M / sec, "normwise_vs_n1_fp64": err_of(out),
                        "vs_n1_same_form": res[form]["seconds"] / sec, "err_bound_normwise_vs_fp64_n2": bounds[form]}
    try:
        orc = oracle_kernel_rate(w)
    except Exception as e:  # the timing is context; the GPU numbers stand without it
        orc = {"unavailable": str(e)[:200]}
    return {"workload": f"{w.name}, all {w.n_x} cells, n_M = {w.n_M}", "forms": res, "oracle_fp64": orc,
            "fp64_sliding_window": {"seconds": dft_sec, "cellM_per_s": w.n_x * w.n_M / dft_sec,
                                    "note": "wmc_kernel_eval_dft, the reference of err_measured_normwise"},
            "n2_network": {"note": "N = 2 barycentric network of Sec. 2.3 (h pair terms against the N = 1 form's "
                                   "h - 1 folded differences); errors against the FP64 N = 2 oracle",
                           "forms": n2}}


def n2_train_rate(wmc, torch, dev, stream, n_examples=100, epochs=200, n_runs=152):
    """The trained N = 2 network (Sec. 2.3): 100 Gaussian-bump potentials on
    256 cells (Q = n_M = 64), 200 epochs of SGD (one example per step), a sweep
    of n_runs learning rates log-spaced over [1e-5, 1e-2] (the paper's 1e-5,
    1e-4, 1e-3 among them), one thread block per run, all in one launch; the
    exact kernels from wmc_kernel_eval_rows.  The FP64 oracle's SGD step is
    timed on a bounded sample of steps."""
    from paper_1806_00082_gb300 import n2train
    w = wi.N2_TRAIN
    p = wmc.Params.of(w)
    ws = wmc.workspace(p, dev)
    Vs = torch.from_numpy(wi.gaussian_bumps(n_examples, n_x=w.n_x)).to(dev)
    order = torch.from_numpy(wi.sgd_order(epochs, n_examples)).to(dev)
    lrs = torch.logspace(-5, -2, n_runs, device=dev)
    for k, v in enumerate((1e-5, 1e-4, 1e-3)):  # the paper's three rates as exact values
        lrs[int(round((math.log10(v) + 5) / 3 * (n_runs - 1)))] = v
    with torch.cuda.stream(stream):
        wmc.init(p, ws)
        n2train.train(p, Vs, order[:2], lrs, ws)  # warm-up
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        params, loss = n2train.train(p, Vs, order, lrs, ws)
        e1.record(stream)
        stream.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3
    h = w.Q // 2
    steps = n_runs * epochs * n_examples
    terms = steps * w.n_x * h * h * 3.0  # model terms per step: forward + the two gradient sums
    by_lr = {}
    for v in (1e-5, 1e-4, 1e-3):
        r = int(round((math.log10(v) + 5) / 3 * (n_runs - 1)))
        by_lr[f"{v:g}"] = {"loss_first_epoch": float(loss[r, 0]), "loss_last_epoch": float(loss[r, -1])}
    orc = {}
    try:
        import oracle
        from oracle import n2train as nt
        po = oracle.params(w)
        Vh = Vs.cpu().numpy()
        T = np.stack([oracle.kernel_rows(po, Vh[e], np.arange(w.n_x))[:, w.Q // 2:] for e in range(4)]) * nt.target_scale(w.Q)
        prm = nt.initial_params(w.Q)
        t0 = time.perf_counter()
        n_s = 0
        while time.perf_counter() - t0 < 5.0:
            _, g = nt.loss_and_grad(prm, Vh[n_s % 4], T[n_s % 4], w.Q)
            prm = prm - 1e-4 * g
            n_s += 1
        orc = {"sgd_steps_per_s": n_s / (time.perf_counter() - t0), "cores": 1, "sample": f"{n_s} SGD steps, FP64 numpy"}
    except Exception as e:  # the timing is context; the GPU numbers stand without it
        orc = {"unavailable": str(e)[:200]}
    return {"workload": f"{w.name}: {n_examples} Gaussian bumps, {epochs} epochs, {n_runs} learning rates",
            "seconds": sec, "sgd_steps_per_s": steps / sec, "model_terms_per_s": terms / sec,
            "paper_learning_rates": by_lr, "oracle_fp64": orc}


def drift_only_rate(wmc, torch, dev, stream, flush, steps=20, warmup=4):
    """Secondary leg, labelled drift-only: the 2000-cell barrier with 1e7
    particles, whose packet starts farther than L_C / 2 from the barrier, so
    its first steps create no pairs (drift, absorption and the histogram only)."""
    w = wi.BARRIER_2000
    p = wmc.Params.of(w)
    V = torch.from_numpy(wi.potential(w)).to(dev)
    a = torch.from_numpy(wi.initial_histogram(w)).to(dev)
    b = torch.empty_like(a)
    ws = wmc.workspace(p, dev)
    tot = 0.0
    with torch.cuda.stream(stream):
        wmc.init(p, ws)
        wmc.run(p, V, a, b, 1, warmup, ws)
        wmc.reset_counters(p, ws)
        t = 1 + warmup
        for _ in range(steps // 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wmc.run(p, V, a, b, t, 2, ws)
            e1.record(stream)
            stream.synchronize()
            tot += e0.elapsed_time(e1) * 1e-3
            t += 2
        c = wmc.get_counters(p, ws)
    return {"workload": f"{w.name} (drift-only: no pairs in these steps)", "value": c["particle_steps"] / tot,
            "unit": UNIT, "steps": 2 * (steps // 2), "ms_per_step": 1e3 * tot / (2 * (steps // 2)),
            "pairs": c["pairs"]}


def batched_rate(wmc, torch, dev, stream, n_sims=512, steps=20, warmup=2):
    """The batched form: n_sims independent barrier simulations (per-simulation
    draws, seed 2), all advanced by one launch per phase; particle-steps/s over
    the batch, work-item size from the autotuner."""
    wls = wi.batch_workloads(n_sims, seed=2)
    ps = wmc.params_array([wmc.Params.of(w) for w in wls])
    co, ho = wmc.batch_layout(ps)
    V = torch.from_numpy(np.concatenate([wi.potential(w) for w in wls])).to(dev)
    H = torch.from_numpy(np.concatenate([wi.initial_histogram(w).reshape(-1) for w in wls])).to(dev)
    ws = wmc.batch_workspace(ps, dev)
    b = torch.empty_like(H)
    with torch.cuda.stream(stream):
        wmc.batch_init(ps, ws)
        per = wmc.batch_autotune(ps, V, H, b, 1, ws)
        wmc.batch_run(ps, V, H, b, 1, 2 * warmup, ws, per_thread=per)
        wmc.batch_init(ps, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wmc.batch_run(ps, V, H, b, 1 + 2 * warmup, steps, ws, per_thread=per)
        e1.record(stream)
        stream.synchronize()
        c = wmc.batch_get_counters(ps, ws)
    sec = e0.elapsed_time(e1) * 1e-3
    return {"workload": f"{n_sims} barrier simulations, cells U[200,4000], n_M in {{128,256}}, N0 U[1e4,1e6]",
            "value": c["particle_steps"] / sec, "unit": UNIT, "steps": steps, "ms_per_step": 1e3 * sec / steps,
            "cells": co[-1], "particles_at_start": int(sum(w.packet.n0 for w in wls)), "per_thread": per,
            "pairs": c["pairs"], "flags": c["flags"]}


def adjoint_rate(wmc, torch, dev, stream, n_pot=64, reps=5):
    """The differentiation form on 64 tanh-barrier potentials x 4096 cells
    (Q = 256, n_M = 512): forward (potential, kernel rows, gamma) and backward
    (kernel adjoint, potential adjoint), timed with events."""
    from paper_1806_00082_gb300.adjoint import kernel_of_potential
    w = wi.TANH_BARRIERS_4096
    p = wmc.Params.of(w)
    ws = wmc.workspace(p, dev)
    theta0 = torch.from_numpy(wi.tanh_parameters(n_pot, n_x=w.n_x, dx_nm=w.dx_m * 1e9)).to(dev)
    g = torch.randn((n_pot * w.n_x, w.Q // 2), device=dev, generator=torch.Generator(dev).manual_seed(0)) * 1e-15
    gg = torch.randn(n_pot * w.n_x, device=dev, generator=torch.Generator(dev).manual_seed(1)) * 1e-16
    fw, bw = 0.0, 0.0
    with torch.cuda.stream(stream):
        wmc.init(p, ws)
        for r in range(reps + 2):
            theta = theta0.clone().requires_grad_(True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            VWh, gamma = kernel_of_potential(theta, p, 16, 16, 0.5, ws)
            loss = (VWh * g).sum() + (gamma * gg).sum()
            e1.record(stream)
            loss.backward()
            e2.record(stream)
            stream.synchronize()
            if r >= 2:
                fw += e0.elapsed_time(e1) * 1e-3
                bw += e1.elapsed_time(e2) * 1e-3
    h = w.Q // 2
    flops = 2.0 * n_pot * w.n_x * (h - 1) ** 2
    # the kernel adjoint alone (wmc_kernel_vjp: the Abar contraction on the
    # tensor cores, 3xTF32, then the scatter to Vbar), L2 flushed before each call
    with torch.cuda.stream(stream):
        VWh, _ = kernel_of_potential(theta0.clone(), p, 16, 16, 0.5, ws)
        VWh = VWh.detach().contiguous()
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        vjp = 0.0
        for r in range(reps + 2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wmc.kernel_vjp(p, VWh, g, gg, n_pot, ws)
            e1.record(stream)
            stream.synchronize()
            if r >= 2:
                vjp += e0.elapsed_time(e1) * 1e-3
        vjp /= reps
    peaks, src = _peaks()
    issued = 3.0 * 2.0 * n_pot * w.n_x * h * h  # three TF32 products over the padded h x h contraction
    peak_tf32 = peaks["bf16_tflops"] * 1e12 * (1.1 / 2.25)
    return {"workload": f"{n_pot} potentials x {w.n_x} cells, Q = {w.Q}, n_M = {w.n_M}, 64 parameters each",
            "forward_s": fw / reps, "backward_s": bw / reps,
            "forward_tflops_algorithmic": flops / (fw / reps) / 1e12,
            "backward_tflops_algorithmic": flops / (bw / reps) / 1e12,
            "kernel_vjp_s": vjp,
            "kernel_vjp_roofline": {"bound": "tensor", "achieved": issued / vjp / 1e12, "peak": peak_tf32 / 1e12,
                                    "unit": "TFLOP/s", "frac": issued / vjp / peak_tf32, "traffic": None,
                                    "peak_source": f"{src} bf16 dense x 1.1/2.25 (nominal tf32/bf16)",
                                    "note": "lower bound: the time includes the CUDA-core scatter to Vbar"},
            "grad_err_bound_normwise": 1e-4}


def single_leg(args):
    """One secondary leg on cuda:0, printed as its own JSON object (profiling aid)."""
    import torch
    from paper_1806_00082_gb300 import build, wmc
    build.build()
    wmc.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    if args.leg == "kernel":
        out = kernel_eval_rate(wmc, torch, dev, stream, flush, reps=max(1, args.steps))
    elif args.leg == "drift":
        out = drift_only_rate(wmc, torch, dev, stream, flush)
    elif args.leg == "n2train":
        out = n2_train_rate(wmc, torch, dev, stream)
    elif args.leg == "batched":
        out = batched_rate(wmc, torch, dev, stream, steps=max(2, args.steps), warmup=1)
    else:
        out = adjoint_rate(wmc, torch, dev, stream, reps=max(1, args.steps))
    print(json.dumps({"leg": args.leg, **out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="double-barrier-16384", choices=sorted(wi.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the secondary legs (kernel, drift-only, "
                    "batched, adjoint)")
    ap.add_argument("--leg", default="all", choices=["all", "kernel", "drift", "batched", "adjoint", "n2train"],
                    help="run one secondary leg alone (for profiling); 'all' is the benchmark")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = wi.WORKLOADS[args.workload]
    if args.impl == "reference":
        return reference_arm(args, w)
    if args.leg != "all":
        return single_leg(args)
    return native_arm(args, w)


if __name__ == "__main__":
    sys.exit(main())
