"""Benchmark: cell-sweep updates/s of the persistent load-balanced step on one
GB300 (or N independent replicas), with roofline, clocks, end-to-end and
CPU-oracle baselines.

One benchmark step = one rebalance period: `period` time steps of every VP
(advection, k_c Thomas sweeps, store, global sum, per-VP cost stamps, grid
barrier) in one persistent launch, then the load measurement and the
rebalance.  The headline strategy is greedy_blocked+steal+dev+pred+thr:
the measured costs (Sec. V) feed GreedyLB applied block by block to the VPs
in spatial order (each processor takes one VP of every block of nprocs,
heaviest to least loaded); processors that finish early take items of the
processor with the most left; measurement and balancer run as device
kernels behind the step launch (no host round trip); at a k_c re-draw the
costs are rescaled for the new array before the balancer runs; and the
table is kept while its predicted max/mean stays within 1.15.  The static
table, the paper's GreedyLB-then-RefineSwapLB schedule, its spatial
variant and the atomic queue, with host or device balancing, are measured
the same way and reported beside it.  The k_c array is re-drawn every 50
time steps as the workload prescribes.

Strategy names: an lb_strategy name, optionally followed by "+steal"
(end-of-step work stealing), "+dev" (device balancer), "+pred" (cost
rescale at k_c re-draws, with +dev), "+thr" (keep a table within the
1.15 threshold, with +dev) and "+graph" (each period one CUDA graph
replay: steps, device measurement, device rebalance; with +dev); kernel
choices "+pair" (split columns on paired warps), "+half" (on half-warps),
"+twin" (one lane per column, packed twisted halves), "+tma" (TMA-staged)
and "+one" (one lane per column, plain Thomas) override the default, which
takes twin halves where at least 3/4 of the columns lie in VPs whose width is
a multiple of 16, or the grid runs the Jacobi sweep (and the FP32 pivots are
constant from level 8 on), and half-warps otherwise.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--period P] [--strategy auto|static|queue|...]

Prints one JSON line (rank 0).  The default workload's fields (403 MB each)
exceed the 129 MB L2, so no flush is needed between timed steps.
"""
import argparse
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

DEFAULT_WORKLOAD = "lognormal_fp32_1024x1024x96"
SIZEOF = {"f64": 8, "f32": 4, "bf16": 2}
# ctxs of the end-to-end leg: while one computes, the copy engines upload the
# next one's input and download the last one's result (three, so that a ctx's
# download and its next upload need not wait on each other)
E2E_RING = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--period", type=int, default=10)
    ap.add_argument("--strategy", default="greedy_blocked+steal+dev+pred+thr")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--threads", type=int, default=0, help="threads per processor (0: default)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the side-by-side runs of the other strategies")
    ap.add_argument("--measure-study", action="store_true",
                    help="instead of the benchmark: per-VP costs measured concurrently with 1, 2 "
                         "or 4 processors per SM and in serialized steps, how well each balances, "
                         "and the throughput the serialized steps cost")
    ap.add_argument("--shard-study", action="store_true",
                    help="instead of the benchmark: a sharded run of two ranks emulated on one "
                         "GPU (two ctxs, halo columns packed and unpacked every step): each "
                         "rank's step, the exchange per step and its bytes, and the assembled "
                         "field against one ctx")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region:
    one sample every 10 ms, each stamped with the host time it arrived; only
    the samples inside the timed window count (the GPU runs the enqueued work
    between the start of the window and the final synchronize)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self, window=None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.summarise(self.lines, window)

    @staticmethod
    def summarise(stamped, window=None):
        """Median SM clock, highest max clock and active throttle reasons of
        the (host time, csv line) samples inside window (all samples when
        none fell inside: a window shorter than one interval)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = stamped
        if window:
            inside = [(t, l) for t, l in stamped if window[0] <= t <= window[1]]
            lines = inside or stamped
        for _, l in lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "samples_in_timed_window": (sum(1 for t, _ in stamped
                                                if window[0] <= t <= window[1])
                                            if window else None)}

def epochs_needed(nsteps_total, epoch_steps):
    """Re-draw epochs a run of nsteps_total time steps can ask for: every
    step t < nsteps_total runs under epoch t // epoch_steps, and the balancer
    call after the last step may install the array of the step that would
    come next, epoch nsteps_total // epoch_steps (with "+pred" the new array
    is installed before the balancer runs)."""
    if not epoch_steps:
        return range(0)
    return range(nsteps_total // epoch_steps + 1)


def kc_epochs(w, nsteps_total):
    """Device-independent k_c arrays for every re-draw epoch the run touches."""
    return {e: [w.kc_array(gi, e) for gi in range(len(w.grids))]
            for e in epochs_needed(nsteps_total, w.kc_epoch_steps)}


def total_time_steps(args, ring=None):
    """Time steps any one ctx of the run executes at most: warm-up and timed
    periods of the headline ctx plus its share of the end-to-end periods
    (the end-to-end ring's other ctxs run fewer)."""
    ring = ring or E2E_RING
    return (args.warmup + args.steps + (args.steps + ring - 1) // ring) * args.period


def bench_config(w, args, world):
    """The workload as both arms name it (no run-dependent values)."""
    return {"workload": w.name, "global_batch": len(w.grids), "period_steps": args.period,
            "time_steps_per_step": args.period, "vps": len(w.vps), "cells": w.cells,
            "strategy": args.strategy, "parallelism": "replicas" if world > 1 else "1gpu",
            "l2": "fields larger than L2 (no flush)"}


def max_over_ranks(x):
    """Largest value over all ranks (time-like quantities); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x):
    """Sum over all ranks (work done by independent replicas)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(work_local, ms_local):
    """Whole-job throughput of N replicas: all ranks' work over the slowest
    rank's time (the barrier-bracketed region)."""
    return sum_over_ranks(work_local) / (max_over_ranks(ms_local) / 1000.0)


def roofline_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_traffic(kernel_tag):
    """Per-launch DRAM bytes of the timed kernel from a committed ncu summary,
    valid only while the kernel sources are unchanged (hash recorded)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        from paper_1310_4218_gb300.build import source_hash
        e = d.get(kernel_tag)
        if e and e.get("source_hash") == source_hash():
            return e
    except Exception:
        pass
    return None


def cpu_oracle_rate(w, budget_s=12.0):
    """The FP64 oracle as it stands (single thread) on a bounded sample of the
    workload: a periodic sub-grid of whole columns (side <= 96) with the
    workload's k_c values over that patch, stepped until the budget is used.
    Returns (cell-sweep updates/s, description, steps, seconds)."""
    import oracle
    g = w.grids[0]
    side = min(g.nx, g.ny, 96)
    epochs = kc_epochs(w, 1)
    if g.kc_disk:
        kc = oracle.kc_field(oracle.OracleGrid.from_spec(g), 0)
    else:
        kc = epochs[0][0]
    # the patch with the largest total k_c among a few candidates, so the
    # sample carries the workload's mean load or more
    best, patch = -1, None
    for y0 in range(0, g.ny - side + 1, max(side, (g.ny - side) // 4 or 1)):
        for x0 in range(0, g.nx - side + 1, max(side, (g.nx - side) // 4 or 1)):
            s_ = int(kc[y0:y0 + side, x0:x0 + side].sum())
            if s_ > best:
                best, patch = s_, (x0, y0)
    x0, y0 = patch
    kcp = np.ascontiguousarray(kc[y0:y0 + side, x0:x0 + side], dtype=np.int32)
    og = oracle.OracleGrid(side, side, g.nz, g.cx, g.cy, g.cz, g.r, False, (0, 0, 0, 0, 0),
                           1, 1, kcp, getattr(g, "dynamics", 0), getattr(g, "nu", 1.0 / 7.0))
    q = np.ascontiguousarray(g.initial_field()[:, y0:y0 + side, x0:x0 + side])
    per_step = int(kcp.sum(dtype=np.int64)) * g.nz
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        q, _ = oracle.run(og, q, 1, t0=steps)
        steps += 1
    dt = time.perf_counter() - t0
    desc = ("%d steps of a periodic %dx%dx%d patch (k_c from %s at (%d,%d)), one thread"
            % (steps, side, side, g.nz, w.name, x0, y0))
    return per_step * steps / dt, desc, steps, dt


def _oracle_worker(job):
    """One single-threaded oracle run (spawned process): (workload, budget)."""
    name, budget_s = job
    from workloads import get_config
    v, _, steps, dt = cpu_oracle_rate(get_config(name), budget_s)
    return v, steps, dt


def cpu_oracle_rate_all_cores(w, budget_s=8.0):
    """The same bounded sample on every host core at once: one unmodified,
    single-threaded oracle per core (a spawned process pool, so that no
    process is forked after CUDA was initialised), each stepping its own copy
    of the patch.  Returns the summed rate and the core count, or an error
    string instead of failing the benchmark."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_worker, [(w.name, budget_s)] * n)
        return {"value": sum(r[0] for r in res), "unit": "cell-sweep updates/s", "cores": n,
                "sample": "%d processes, each as the one-thread sample (%d-%d steps)"
                          % (n, min(r[1] for r in res), max(r[1] for r in res))}
    except Exception as ex:                      # reported, never fatal
        return {"value": None, "cores": n, "error": repr(ex)[:200]}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, timed on the host cores."""
    from workloads import get_config
    w = get_config(args.workload)
    if rank != 0:
        return
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_rate(w, budget_s=1.0)
    vals, times = [], []
    for _ in range(args.steps):
        v, desc, steps, dt = cpu_oracle_rate(w, budget_s=max(2.0, 30.0 / max(args.steps, 1)))
        vals.append(v)
        times.append(dt)
    value = float(np.median(vals))
    out = {"metric": "cell-sweep updates/s", "value": value, "unit": "cell-sweep updates/s",
           "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1000.0 * float(np.median(times)), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(w, args, world),
           "cpu_baseline": {"value": value, "unit": "cell-sweep updates/s", "cores": 1,
                            "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": "cell-sweep updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


class StrategyRun:
    """One ctx on the workload, driven period by period with one strategy."""

    def __init__(self, w, fields, epochs, kc_dev, args, dev, stream, strategy):
        from paper_1310_4218_gb300 import lb
        from paper_1310_4218_gb300.sim import Simulation
        self.lb, self.w, self.epochs, self.kc_dev = lb, w, epochs, kc_dev
        # "<strategy>[+steal][+dev]": +steal, processor tables with end-of-step
        # work stealing; +dev, measurement and balancer on the device
        parts = strategy.split("+")
        strategy, flags = parts[0], set(parts[1:])
        steal = "steal" in flags
        self.dev_mode = "dev" in flags
        # kernel choice (default: twin halves where VP widths allow, else
        # half-warps): "+tma" TMA-staged, "+half" / "+pair" split columns on
        # half-warps / paired warps
        staged = "tma" in flags
        half = "half" in flags
        pair = "pair" in flags
        one = "one" in flags          # "+one": one lane per column
        twin = "twin" in flags        # "+twin": one lane per column, packed halves
        # "+df": the dataflow kernel (no grid barrier between steps) where it
        # applies: the atomic queue on the exact-nz twin kernels
        dataflow = "df" in flags
        # "+pred": at a k_c re-draw the new array is installed before the
        # balancer runs and the costs are rescaled by the fitted model
        self.predict = "pred" in flags and self.dev_mode
        self.threshold = "thr" in flags and self.dev_mode
        # "+graph": each period replays one CUDA graph (steps, device
        # measurement, device rebalance); k_c re-draws between replays
        self.use_graph = "graph" in flags and self.dev_mode and strategy != "queue"
        self.gexec = None
        self.kc_epoch = None
        self.dev_tags = []
        self.kernels = 0             # our kernel launches (step, k_c switch, balancer)
        self.P, self.strategy, self.dev, self.stream = args.period, strategy, dev, stream
        opt = lb.lb_default_options()
        opt.threads_hint = args.threads
        opt.queue_order = 0
        opt.steal = 1 if steal else 0
        opt.predict_kc = 1 if self.predict else 0
        opt.staged_loads = 1 if staged else 0
        if half:
            opt.threads_hint = 2
        if pair:
            opt.threads_hint = 3
        if one:
            opt.threads_hint = 1
        if twin:
            opt.threads_hint = 4
        opt.dataflow = 1 if dataflow else 0
        kc0 = [epochs[0][gi] for gi in range(len(w.grids))] if epochs else None
        self.sim = Simulation(w.grids, fields, w.vps, kc_arrays=kc0, options=opt, device=dev,
                              stream=stream)
        self.info = self.sim.info()
        self.t = 0
        self.stats = {}
        self.timed_rows = []
        self.name = strategy if not flags else "+".join([strategy] + parts[1:])

    def launches(self, t0, t1):
        """Time steps t0..t1-1 as persistent launches, split where the k_c
        array is re-drawn.  Returns the number of launches."""
        t, n_launch = t0, 0
        w = self.w
        while t < t1:
            n = t1 - t
            if self.epochs:
                e = t // w.kc_epoch_steps
                self.set_epoch(e)
                n = min(n, (e + 1) * w.kc_epoch_steps - t)
            if self.use_graph and n == self.P:
                if self.gexec is None:
                    self.gexec = self.lb.lb_graph_create_periods(
                        self.sim.ctx, self.P, self.strategy, 1, 1.15 if self.threshold else 0.0)
                self.lb.lb_graph_launch(self.sim.ctx, self.gexec)
                self.kernels += 4                  # measure, prep, balance, items
                self.dev_tags.append("graph")
            else:
                self.sim.step(n)
            t += n
            n_launch += 1
        self.kernels += n_launch
        return n_launch

    def set_epoch(self, e):
        """Install the k_c arrays of epoch e (once)."""
        if e == self.kc_epoch:
            return
        if e not in self.kc_dev:
            raise KeyError("k_c epoch %d was not drawn (epochs 0..%d)" % (e, max(self.kc_dev)))
        for gi in range(len(self.w.grids)):
            self.lb.lb_set_kc(self.sim.ctx, gi, self.kc_dev[e][gi].data_ptr())
            self.kernels += 4 if self.predict else 1   # switch, features, fit, rescale
        self.kc_epoch = e

    def balance(self, tag, t_next):
        """Load measurement (Sec. V) and the balancer call (Sec. VI) before
        time step t_next."""
        if self.use_graph and self.gexec is not None:
            # measured and rebalanced inside the graph; a k_c re-draw with
            # +pred rescales the costs and forces one more rebalance now
            if self.dev_tags and self.dev_tags[-1] == "graph":
                self.dev_tags[-1] = tag
            if self.predict and self.epochs:
                e = t_next // self.w.kc_epoch_steps
                if e != self.kc_epoch:
                    self.set_epoch(e)
                    self.lb.lb_device_rebalance_if(self.sim.ctx, self.strategy,
                                                   1.15 if self.threshold else 0.0)
                    self.kernels += 3
                    self.dev_tags.append(tag)
            return
        if self.dev_mode:
            # enqueued only: measurement, cost rounding and ranks, balancer,
            # table kernels (the queue has no table: measurement and record)
            self.lb.lb_device_measure(self.sim.ctx)
            if self.predict and self.epochs:
                self.set_epoch(t_next // self.w.kc_epoch_steps)
            if self.strategy == "queue" and self.info.strategy != self.lb.LB_ATOMIC_QUEUE:
                self.sim.rebalance("queue")       # enter queue mode once
                self.info = self.sim.info()
            # "+thr": keep the table while its predicted max/mean <= 1.15
            self.lb.lb_device_rebalance_if(self.sim.ctx, self.strategy,
                                           1.15 if self.threshold else 0.0)
            self.kernels += 3 if self.strategy == "queue" else 4
            self.dev_tags.append(tag)
            return
        cost, busy = self.sim.measure()
        used = busy[busy > 0]
        st = {"sm_max_over_mean": float(used.max() / used.mean()) if used.size else None}
        mean = float(cost.sum()) / self.info.nprocs
        st["granularity_floor"] = float(max(cost.max(), mean) / mean) if mean > 0 else None
        if self.strategy != "static":
            mig, pred = self.sim.rebalance(self.strategy)
            st["migrations"] = mig
            st["predicted_max_over_mean"] = pred
        self.record(tag, st)

    def record(self, tag, st):
        """Keep one period's balance record: the latest under its tag, and
        every timed one in order."""
        self.stats[tag] = st
        if tag == "timed":
            self.timed_rows.append(st)

    def collect(self):
        """Device mode: per-period records from the balance history."""
        if not self.dev_mode or not self.dev_tags:
            return
        rows = self.lb.lb_balance_history(self.sim.ctx)[-len(self.dev_tags):]
        for tag, r in zip(self.dev_tags, rows):
            self.record(tag, {"sm_max_over_mean": float(r[4]), "granularity_floor": float(r[5]),
                              "migrations": int(r[2]), "predicted_max_over_mean": float(r[3])})
        self.dev_tags = []

    def imbalance_summary(self):
        """SM max/mean over the timed periods (mean and worst), the first
        (static) period's, the granularity floor and the balancer's
        predicted max/mean, from the per-period records."""
        rows = [r for r in self.timed_rows if r.get("sm_max_over_mean") is not None]
        out = {"strategy": self.name, "periods": len(rows)}
        if rows:
            sm = [r["sm_max_over_mean"] for r in rows]
            out["sm_max_over_mean"] = float(np.mean(sm))
            out["sm_max_over_mean_worst"] = float(np.max(sm))
            fl = [r["granularity_floor"] for r in rows if r.get("granularity_floor")]
            out["granularity_floor"] = float(np.max(fl)) if fl else None
            pr = [r["predicted_max_over_mean"] for r in rows
                  if r.get("predicted_max_over_mean") is not None]
            out["predicted_max_over_mean"] = float(np.mean(pr)) if pr else None
        first = self.stats.get("first", {})
        out["first_period_sm_max_over_mean"] = first.get("sm_max_over_mean")
        return out

    def warmup(self, nper):
        import torch
        for wi in range(nper):
            self.launches(self.t, self.t + self.P)
            self.t += self.P
            self.balance("first" if wi == 0 else "warmup", self.t)
        torch.cuda.synchronize(self.dev)
        self.collect()

    def timed(self, nper, sampler=None):
        """nper periods between CUDA events; returns the measurement."""
        import torch
        lb, stream = self.lb, self.stream
        sw0, cs0 = lb.lb_work_done(self.sim.ctx)
        torch.cuda.synchronize(self.dev)
        k0 = self.kernels
        if sampler:
            sampler.start()
            time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kev = []
        w0 = time.monotonic()
        e0.record(stream)
        for _ in range(nper):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nl = self.launches(self.t, self.t + self.P)
            b.record(stream)
            kev.append((a, b, nl))
            self.balance("timed", self.t + self.P)
            self.t += self.P
        e1.record(stream)
        torch.cuda.synchronize(self.dev)
        w1 = time.monotonic()
        clocks = sampler.stop((w0, w1)) if sampler else None
        sw1, cs1 = lb.lb_work_done(self.sim.ctx)
        self.collect()
        return {"ms": e0.elapsed_time(e1), "sweeps": sw1 - sw0, "cells": cs1 - cs0,
                "kernel_ms": [a.elapsed_time(b) / n for a, b, n in kev],
                "launches": sum(n for _, _, n in kev), "kernels": self.kernels - k0,
                "clocks": clocks}

    def close(self):
        if self.gexec is not None:
            self.lb.lb_graph_destroy(self.sim.ctx, self.gexec)
            self.gexec = None
        self.sim.close()


def end_to_end(ring, fields, nper, stream, dev):
    """The benchmark step through the public API with host buffers.  Period n
    runs on ctx n mod len(ring); all ctxs share one compute stream.  A
    period's input is copied host -> device (pinned) on an upload stream
    once that ctx's previous result has left the device, the period computes
    after its upload, and its result is copied device -> host on a download
    stream, so uploads and downloads for the other ctxs overlap the period
    that computes.  Every copy and every period lies inside the timed
    region (events on the compute stream, which waits for the last
    download).  Returns the rate and the bytes each period copies."""
    import torch
    w = ring[0].w
    if not all(g.storage == "f32" for g in w.grids):
        return None
    h_in = [torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).pin_memory()
            for f in fields]
    h_out = [torch.empty_like(x).pin_memory() for x in h_in]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    s0 = [r.lb.lb_work_done(r.sim.ctx)[0] for r in ring]
    k0 = [r.kernels for r in ring]
    freed = [None] * len(ring)
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    up.wait_stream(stream)
    down.wait_stream(stream)
    for n in range(nper):
        x = n % len(ring)
        r = ring[x]
        if freed[x] is not None:
            up.wait_event(freed[x])
        with torch.cuda.stream(up):
            for gi in range(len(w.grids)):
                r.sim.field_tensor(gi).copy_(h_in[gi], non_blocking=True)
        loaded = torch.cuda.Event()
        loaded.record(up)
        stream.wait_event(loaded)
        r.launches(r.t, r.t + r.P)
        r.balance("e2e", r.t + r.P)
        r.t += r.P
        done = torch.cuda.Event()
        done.record(stream)
        down.wait_event(done)
        with torch.cuda.stream(down):
            for gi in range(len(w.grids)):
                h_out[gi].copy_(r.sim.field_tensor(gi), non_blocking=True)
        freed[x] = torch.cuda.Event()
        freed[x].record(down)
    stream.wait_stream(up)
    stream.wait_stream(down)
    c1.record(stream)
    torch.cuda.synchronize(dev)
    es = c0.elapsed_time(c1) / 1000.0
    sw = 0
    for r, s in zip(ring, s0):
        r.collect()
        sw += r.lb.lb_work_done(r.sim.ctx)[0] - s
    nbytes = sum(x.numel() * x.element_size() for x in h_in)
    return {"value": sw / es, "unit": "cell-sweep updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "ms_per_step": 1000.0 * es / max(nper, 1), "ctxs": len(ring),
            "kernels": sum(r.kernels for r in ring) - sum(k0)}


def item_work_model(w, info, kc, kappa=6.0):
    """Cost model of the k_c work per VP: nz times the sum over the kernel's
    work items of (kappa + the largest k_c among the item's columns), the
    sweeps a warp runs for the item plus a fixed item overhead."""
    out = np.zeros(len(w.vps))
    iw, ih = info.item_w, info.item_h
    for v, (gi, x0, y0, ww, hh) in enumerate(w.vps):
        b = kc[y0:y0 + hh, x0:x0 + ww]
        if ih == 0:
            f = b.ravel()
            mx = [f[c:c + iw].max() for c in range(0, f.size, iw)]
        else:
            mx = [b[ty:ty + ih, tx:tx + iw].max() for ty in range(0, hh, ih) for tx in range(0, ww, iw)]
        out[v] = (kappa * len(mx) + float(np.sum(mx))) * w.grids[gi].nz
    return out


def measurement_study(args):
    """Sec. V measures each VP's load in serialized steps because concurrent
    GPU work timed unreliably on the paper's hardware (Table I).  Here: the
    per-VP costs measured concurrently with 1, 2 and 4 processors (CTAs)
    sharing each SM, and in serialized steps (one working warp per
    processor); each cost vector's correlation with the serialized one and
    with the k_c work model; the SM max/mean and kernel time of a period
    balanced (blocked GreedyLB) on each; and what measuring in serialized
    steps would cost the schedule."""
    import torch

    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    from workloads import get_config

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    w = get_config(args.workload)
    P = args.period
    kc = [w.kc_array(gi, 0) for gi in range(len(w.grids))] if w.kc_epoch_steps else None
    fields = [g.initial_field() for g in w.grids]

    def make(ctas=1):
        o = lb.lb_default_options()
        o.ctas_per_sm = ctas
        return Simulation(w.grids, fields, w.vps, kc_arrays=kc, options=o, device=dev,
                          stream=stream)

    def timed(fn):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    costs, ms, infos = {}, {}, {}
    for mode, ctas, serial in (("concurrent, 1 processor/SM", 1, False),
                               ("concurrent, 2 processors/SM", 2, False),
                               ("concurrent, 4 processors/SM", 4, False),
                               ("serialized steps", 1, True)):
        sim = make(ctas)
        infos[mode] = sim.info()
        sim.step(P)
        sim.measure()
        if serial:
            ms[mode] = timed(lambda: lb.lb_step_serial(sim.ctx, P)) / P
        else:
            ms[mode] = timed(lambda: sim.step(P)) / P
        costs[mode] = sim.measure()[0]
        sim.close()
    ref = costs["serialized steps"]
    model = item_work_model(w, infos["concurrent, 1 processor/SM"], kc[0]) if kc else None
    out = {"study": "load measurement under concurrency (Sec. V, Table I)",
           "workload": w.name, "period_steps": P, "modes": {}}
    for mode, c in costs.items():
        row = {"step_ms": ms[mode], "processors": infos[mode].nprocs,
               "threads_per_processor": infos[mode].threads_per_cta,
               "corr_with_serialized": float(np.corrcoef(c, ref)[0, 1]),
               "corr_with_kc_model": float(np.corrcoef(c, model)[0, 1]) if model is not None else None}
        # balance a fresh ctx (1 processor per SM, concurrent) on these costs
        sim = make(1)
        sim.step(P)
        sim.measure()
        sim.set_costs(c)
        sim.rebalance("greedy_blocked")
        row["balanced_period_kernel_ms"] = timed(lambda: sim.step(P))
        _, busy = sim.measure()
        used = busy[busy > 0]
        row["balanced_sm_max_over_mean"] = float(used.max() / used.mean())
        sim.close()
        out["modes"][mode] = row
    tc = ms["concurrent, 1 processor/SM"]
    ts = ms["serialized steps"]
    out["serialized_step_over_concurrent"] = ts / tc
    out["period_time_with_one_serialized_step"] = (ts + (P - 1) * tc) / (P * tc)
    print(json.dumps(out), flush=True)


def shard_study(args, nranks=2, nsteps=20):
    """The sharded run of shard.py (the paper's processors as ranks, Sec. III,
    with the halo exchange of Fig. 2) on one GPU: `nranks` ctxs over the same
    grid, each running the VPs of one 2D block, with the halo columns moved
    by lb_pack_columns / lb_unpack_columns before every step.  The ranks run
    one after the other here, so the numbers are each rank's step and the
    exchange's cost, not a scaling curve; the assembled owned columns must
    equal one ctx running every VP, bit for bit."""
    import time

    import torch

    from paper_1310_4218_gb300 import lb, shard
    from paper_1310_4218_gb300.sim import Simulation
    from workloads import get_config

    dev = torch.device("cuda", 0)
    w = get_config(args.workload)
    kc = [w.kc_array(gi, 0) for gi in range(len(w.grids))] if w.kc_epoch_steps else None
    fields = [g.initial_field() for g in w.grids]

    def make():
        s = Simulation(w.grids, fields, w.vps, kc_arrays=kc, options=lb.lb_default_options(),
                       device=dev)
        s.rebalance("queue")
        return s

    whole = make()
    parts = [make() for _ in range(nranks)]
    st = [shard.GPUStepper(s) for s in parts]
    owner = shard.block_owners(w.vps, w.grids, nranks)
    for r in range(nranks):
        st[r].set_owned((owner == r).astype(np.uint8))
    plans = [shard.HaloPlan(w.vps, w.grids, owner, r, nranks) for r in range(nranks)]

    def exchange():
        for r in range(nranks):
            for (gi, p), cells in plans[r].send.items():
                st[p].unpack(gi, cells, st[r].pack(gi, cells))
        for s in parts:
            s.stream.synchronize()

    def event():
        return torch.cuda.Event(enable_timing=True)

    for _ in range(3):
        exchange()
        for s in st:
            s.step(1)
        whole.step(1)
    torch.cuda.synchronize(dev)
    t_x, t_rank, t_whole = [], [[] for _ in range(nranks)], []
    for _ in range(nsteps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        exchange()
        t_x.append((time.perf_counter() - t0) * 1e3)
        for r in range(nranks):
            a, b = event(), event()
            a.record(parts[r].stream)
            st[r].step(1)
            b.record(parts[r].stream)
            t_rank[r].append((a, b))
        a, b = event(), event()
        a.record(whole.stream)
        whole.step(1)
        b.record(whole.stream)
        t_whole.append((a, b))
    torch.cuda.synchronize(dev)
    equal = True
    for gi, g in enumerate(w.grids):
        ref = whole.field(gi).reshape(g.nz, -1)
        got = np.zeros_like(ref)
        for r in range(nranks):
            cols = np.concatenate([shard.vp_cells(vp, g.nx) for v, vp in enumerate(w.vps)
                                   if owner[v] == r and vp[0] == gi])
            got[:, cols] = parts[r].field(gi).reshape(g.nz, -1)[:, cols]
        equal = equal and bool(np.array_equal(got, ref))
    esize = {"f64": 8, "f32": 4, "bf16": 2}
    halo = [sum(len(c) * w.grids[gi].nz * esize[w.grids[gi].storage]
                for (gi, _), c in plans[r].recv.items()) for r in range(nranks)]
    med = lambda ts: statistics.median(a.elapsed_time(b) for a, b in ts)
    out = {"study": "sharded run, ranks emulated on one GPU (Sec. III, Fig. 2)",
           "workload": w.name, "ranks": nranks, "steps": nsteps,
           "one_ctx_step_ms": med(t_whole),
           "rank_step_ms": [med(t) for t in t_rank],
           "owned_columns": [int(sum(vp[3] * vp[4] for v, vp in enumerate(w.vps) if owner[v] == r))
                             for r in range(nranks)],
           "halo_bytes_received_per_step": halo,
           "exchange_ms_per_step": statistics.median(t_x),
           "assembled_field_equals_one_ctx": equal}
    for s in parts + [whole]:
        s.close()
    print(json.dumps(out), flush=True)


COMPARED = ("static", "static+steal", "auto", "auto+dev", "auto_spatial+steal",
            "auto_spatial+steal+dev", "greedy_blocked+dev", "greedy_blocked+dev+pred",
            "greedy_blocked+dev+pred+thr", "greedy_blocked+steal+dev",
            "greedy_blocked+steal+dev+pred", "greedy_blocked+steal+dev+pred+thr",
            "greedy_blocked+steal+dev+pred+thr+graph", "greedy_blocked+steal+dev+pred+thr+pair",
            "greedy_blocked+steal+dev+pred+thr+twin", "greedy_blocked+steal+dev+pred+thr+tma",
            "queue", "queue+dev", "queue+dev+df")


def main():
    args = parse()
    rank, local_rank, world = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.measure_study:
        if rank == 0:
            measurement_study(args)
        return
    if args.shard_study:
        if rank == 0:
            shard_study(args)
        return

    import torch
    import torch.distributed as dist

    from workloads import get_config

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    w = get_config(args.workload)
    P = args.period
    epochs = kc_epochs(w, total_time_steps(args))
    fields = [g.initial_field() for g in w.grids]
    kc_dev = {e: [torch.as_tensor(a).to(dev) for a in arrs] for e, arrs in epochs.items()}
    stream = torch.cuda.Stream(dev)

    # the headline strategy: device-resident inputs, clocks sampled
    run = StrategyRun(w, fields, epochs, kc_dev, args, dev, stream, args.strategy)
    info = run.info
    run.warmup(args.warmup)
    if world > 1:
        dist.barrier()
    m = run.timed(args.steps, ClockSampler(local_rank))
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(m["ms"])
    s = ms / 1000.0
    value = whole_job_rate(m["sweeps"], m["ms"])
    cells_all = sum_over_ranks(m["cells"])

    g0 = w.grids[0]
    steps_per_launch = args.steps * P / m["launches"]
    bytes_per_step = 2 * w.cells * SIZEOF[g0.storage] + \
        4 * sum(g.nx * g.ny for g in w.grids if not g.kc_disk)
    bytes_per_launch = bytes_per_step * steps_per_launch
    kern_s = statistics.median(m["kernel_ms"]) / 1000.0
    peak, peak_src = roofline_peak()
    achieved = bytes_per_launch / kern_s / 1e9
    tr = load_traffic("lb_step_kernel:%s" % w.name)
    imbalance = run.imbalance_summary()

    e2e = None
    if not args.no_e2e:
        ring = [run]
        try:
            for _ in range(E2E_RING - 1):
                r = StrategyRun(w, fields, epochs, kc_dev, args, dev, stream, args.strategy)
                ring.append(r)
                r.warmup(args.warmup)
            e2e = end_to_end(ring, fields, args.steps, stream, dev)
            if e2e:
                e2e["value"] = sum_over_ranks(e2e["value"])
        except Exception as ex:    # report, keep the device-timed line
            e2e = {"value": None, "unit": "cell-sweep updates/s", "error": repr(ex)[:200]}
        for r in ring[1:]:
            r.close()
    run.close()

    # the other assignments, measured the same way (device-resident inputs):
    # [cell-sweep updates/s, kernel ms per launch, SM max/mean over the timed
    # periods, SM max/mean of the first (static) period]
    compare = {}
    if not args.no_compare:
        for st in [x for x in COMPARED if x != args.strategy]:
            r2 = StrategyRun(w, fields, epochs, kc_dev, args, dev, stream, st)
            r2.warmup(args.warmup)
            m2 = r2.timed(args.steps)
            sm2 = r2.imbalance_summary()
            compare[st] = [m2["sweeps"] / (m2["ms"] / 1000.0),
                           statistics.median(m2["kernel_ms"]),
                           sm2.get("sm_max_over_mean"), sm2.get("first_period_sm_max_over_mean")]
            r2.close()

    cpu = None
    if rank == 0 and not args.no_cpu:
        v, desc, _, _ = cpu_oracle_rate(w)
        cpu = {"value": v, "unit": "cell-sweep updates/s", "cores": 1, "kind": "oracle",
               "sample": desc, "all_cores": cpu_oracle_rate_all_cores(w)}

    if rank == 0:
        # the bulky comparison table first: a reader of the line's tail sees
        # the headline's roofline, imbalance, clocks and end-to-end figures
        out = {
            "strategies_columns": ["updates/s", "kernel ms/launch", "SM max/mean",
                                   "first period SM max/mean"],
            "strategies": compare,
            "metric": "cell-sweep updates/s", "value": value, "unit": "cell-sweep updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if g0.compute == "f32" else "f64",
            "data": "synthetic",
            "config": bench_config(w, args, world),
            "run": {"processors": info.nprocs, "threads_per_cta": info.threads_per_cta,
                    "cell_steps_per_s": cells_all / s,
                    "per_grid_cell_steps_per_s": (
                        [g.nx * g.ny * g.nz * args.steps * P * world / s for g in w.grids]
                        if len(w.grids) > 1 else None)},
            "cpu_baseline": cpu,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "traffic": (tr["dram_bytes_per_step"] * steps_per_launch) if tr else None,
                         "kernel": "lb_step_kernel",
                         "kernel_ms_per_launch": kern_s * 1000.0,
                         "steps_per_launch": steps_per_launch,
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "imbalance": imbalance,
            "clocks": m["clocks"],
            "gpu_launches": m["kernels"],
            "e2e": e2e,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
