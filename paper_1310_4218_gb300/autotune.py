"""Autotuner: picks VP granularity, kernel variant, assignment strategy and
rebalance period for a workload by timing short windows on the device.

Knobs:
  split     -- VP granularity: 1 keeps the layout, 2 cuts every VP of at
               least 2*min_side columns per side into quadrants (finer
               over-decomposition, Sec. III: more, smaller VPs balance better
               but add halo traffic)
  variant   -- lb_options.threads_hint: 0 default kernel, 1 one lane per
               column, 2 split columns on half-warps, 3 on paired warps,
               4 twin halves (one lane per column, packed twisted halves;
               where the pivots do not allow it, half-warps run instead)
  strategy  -- assignment (lb_strategy name), balanced on the device with
               end-of-step stealing, the cost rescale at k_c re-draws and a
               threshold (keep the table while predicted max/mean <= 1.15);
               layouts of more than 8192 VPs use the host balancer
  period    -- time steps between balancer calls

Each candidate runs `warmup` periods, then is timed over `timed` periods
with CUDA events on the ctx stream; the score is cell-sweep updates/s
counted on the device.  Results are cached in a JSON file keyed by a
signature of the workload and the device name.
"""
import hashlib
import itertools
import json
import os

import numpy as np
import torch

from . import lb as L
from .schedule import Schedule
from .sim import Simulation


def split_layout(vps, factor, min_side=8):
    """Cut each VP with w, h >= factor * min_side into factor x factor parts."""
    if factor <= 1:
        return list(vps)
    out = []
    for (g, x0, y0, w, h) in vps:
        if w >= factor * min_side and h >= factor * min_side:
            xs = [x0 + (w * i) // factor for i in range(factor + 1)]
            ys = [y0 + (h * j) // factor for j in range(factor + 1)]
            for j in range(factor):
                for i in range(factor):
                    out.append((g, xs[i], ys[j], xs[i + 1] - xs[i], ys[j + 1] - ys[j]))
        else:
            out.append((g, x0, y0, w, h))
    return out


def signature(grids, vps, kc_epoch_steps):
    """Cache key of a workload: every grid field that changes the kernel, the
    work or the balance (the dynamics and its weight included), the layout
    and the re-draw interval."""
    h = hashlib.sha256()
    for g in grids:
        h.update(repr((g.nx, g.ny, g.nz, g.cx, g.cy, g.cz, g.r, g.storage, g.compute,
                       g.kc_disk, tuple(g.disk), g.k_in, g.k_out,
                       getattr(g, "dynamics", 0), getattr(g, "nu", 1.0 / 7.0))).encode())
    h.update(repr(sorted(vps)).encode())
    h.update(repr(kc_epoch_steps).encode())
    return h.hexdigest()[:16]


def measure(grids, fields, vps, kc_epochs, epoch_steps, strategy, period, variant, warmup=2,
            timed=2, device="cuda:0", threshold=1.15):
    """Cell-sweep updates/s of one configuration (device-timed)."""
    opt = L.lb_default_options()
    opt.threads_hint = variant
    opt.steal = 1
    opt.predict_kc = 1
    kc0 = kc_epochs[0] if kc_epochs else None
    dev = torch.device(device)
    stream = torch.cuda.Stream(dev)
    sim = Simulation(grids, fields, vps, kc_arrays=kc0, options=opt, device=dev, stream=stream)
    try:
        # the device balancer takes up to 8192 VPs; beyond, the host balancer
        dev_ok = len(vps) <= 8192
        sch = Schedule(sim, period, strategy, kc_epochs, epoch_steps,
                       threshold=None if (strategy == "queue" or not dev_ok) else threshold,
                       device=dev_ok)
        for _ in range(warmup):
            sch.run_period()
        torch.cuda.synchronize(dev)
        s0, _ = L.lb_work_done(sim.ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(timed):
            sch.run_period()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        s1, _ = L.lb_work_done(sim.ctx)
        return (s1 - s0) / (e0.elapsed_time(e1) / 1000.0)
    finally:
        sim.close()


def autotune(grids, fields, vps, kc_epochs=None, epoch_steps=0, cache=None,
             strategies=("greedy_blocked", "auto_spatial", "queue"), periods=(10, 20),
             variants=(2, 4),
             splits=(1, 2), device="cuda:0", log=None):
    """Best configuration over the candidate grid; returns a dict with the
    knobs, the score and every candidate's score."""
    key = None
    name = torch.cuda.get_device_name(torch.device(device))
    if cache:
        key = "%s|%s" % (signature(grids, vps, epoch_steps), name)
        if os.path.exists(cache):
            with open(cache) as f:
                d = json.load(f)
            if key in d:
                return d[key]
    scores = []
    for split, variant, strategy, period in itertools.product(splits, variants, strategies,
                                                              periods):
        lay = split_layout(vps, split)
        try:
            v = measure(grids, fields, lay, kc_epochs, epoch_steps, strategy, period, variant,
                        device=device)
        except L.LBError as e:             # e.g. a variant not offered for these grids
            v = None
            if log:
                log("skip %s: %s" % ((split, variant, strategy, period), e))
        scores.append({"split": split, "variant": variant, "strategy": strategy,
                       "period": period, "value": v})
        if log:
            log("split %d variant %d %-12s period %2d: %s" % (split, variant, strategy, period,
                                                            "%.3e" % v if v else "-"))
    ok = [s for s in scores if s["value"]]
    if not ok:
        raise RuntimeError("autotune: no candidate ran on these grids")
    best = max(ok, key=lambda s: s["value"])
    res = dict(best)
    res["candidates"] = scores
    if cache:
        d = {}
        if os.path.exists(cache):
            with open(cache) as f:
                d = json.load(f)
        d[key] = res
        with open(cache, "w") as f:
            json.dump(d, f, indent=1)
    return res
