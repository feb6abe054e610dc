"""The application loop of Fig. 2 on top of a Simulation: runs of `period`
time steps (persistent launches, split where the load array is re-drawn),
each followed by the load measurement (Sec. V) and a balancer call
(Sec. VI; "auto" = GreedyLB on the first call, RefineSwapLB afterwards).
"""
import numpy as np
import torch

from . import lb as L


class Schedule:
    """kc_epochs: {epoch: [int32 (ny, nx) per grid]} for array-k_c grids,
    re-drawn every `epoch_steps` time steps (0: never).

    threshold: if set, the balancer is called only when the measured SM
    max/mean load of the period exceeds it -- the threshold-triggered
    migration the paper plans as future work (Sec. VII): measurements stay
    on (they are free on the device), migrations happen only when needed.

    device: measure and rebalance with the device balancer
    (lb_device_measure / lb_device_rebalance_if): nothing waits for the host
    between periods; per-period records come from lb_balance_history.  A
    threshold then keeps the table while its predicted max/mean under the
    current costs stays within it (on the host balancer the test is on the
    measured SM max/mean).  The atomic queue is entered once on the host.
    With a ctx created with lb_options.predict_kc, the k_c arrays of the
    next segment are installed between the measurement and the balancer
    call, so the balancer sees costs rescaled for the coming array.
    """

    def __init__(self, sim, period, strategy="auto", kc_epochs=None, epoch_steps=0,
                 threshold=None, device=False):
        self.device = device
        self.sim = sim
        self.period = int(period)
        self.strategy = strategy
        self.threshold = threshold
        self.epoch_steps = int(epoch_steps or 0)
        self.kc_dev = {}
        if kc_epochs:
            for e, arrs in kc_epochs.items():
                self.kc_dev[e] = [None if a is None else
                                  torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).to(sim.device)
                                  for a in arrs]
            # the copies ran on torch's current stream; the ctx stream, which
            # may be another one, reads the arrays from the first re-draw on
            torch.cuda.current_stream(sim.device).synchronize()
        self.t = 0
        self.history = []
        self._epoch_set = None

    def _segments(self, t0, t1):
        t = t0
        while t < t1:
            n = t1 - t
            e = None
            if self.epoch_steps:
                e = t // self.epoch_steps
                n = min(n, (e + 1) * self.epoch_steps - t)
            yield t, n, e
            t += n

    def launches_per_period(self, t0=None):
        t0 = self.t if t0 is None else t0
        return sum(1 for _ in self._segments(t0, t0 + self.period))

    def _install(self, e):
        if e is not None and e != self._epoch_set and e in self.kc_dev:
            for gi, d in enumerate(self.kc_dev[e]):
                if d is not None:
                    L.lb_set_kc(self.sim.ctx, gi, d.data_ptr())
            self._epoch_set = e

    def run_steps(self, n):
        """n time steps without a balancer call."""
        for t, m, e in self._segments(self.t, self.t + n):
            self._install(e)
            self.sim.step(m)
        self.t += n

    def balance(self):
        """Measure the loads of the steps since the last call and rebalance."""
        if self.device:
            L.lb_device_measure(self.sim.ctx)
            if self.epoch_steps and getattr(self.sim, "options", None) is not None and \
                    self.sim.options.predict_kc:
                self._install(self.t // self.epoch_steps)
            if self.strategy == "queue" and self.sim.info().strategy != L.LB_ATOMIC_QUEUE:
                self.sim.rebalance("queue")
            L.lb_device_rebalance_if(self.sim.ctx, self.strategy, self.threshold or 0.0)
            rec = {"t": self.t, "device": True}
            self.history.append(rec)
            return rec
        cost, busy = self.sim.measure()
        used = busy[busy > 0]
        rec = {"t": self.t,
               "sm_max_over_mean": float(used.max() / used.mean()) if used.size else None}
        nprocs = self.sim.info().nprocs
        mean = float(cost.sum()) / nprocs
        rec["granularity_floor"] = float(max(cost.max(), mean) / mean) if mean > 0 else None
        skip = (self.threshold is not None and rec["sm_max_over_mean"] is not None
                and rec["sm_max_over_mean"] <= self.threshold)
        rec["rebalanced"] = self.strategy != "static" and not skip
        if rec["rebalanced"]:
            mig, pred = self.sim.rebalance(self.strategy)
            rec["migrations"] = mig
            rec["predicted_max_over_mean"] = pred
        self.history.append(rec)
        return rec

    def device_history(self):
        """Records of the device rebalances (synchronises): dicts with the
        columns of lb.BALANCE_HISTORY_COLUMNS."""
        rows = L.lb_balance_history(self.sim.ctx)
        return [dict(zip(L.BALANCE_HISTORY_COLUMNS, map(float, r))) for r in rows]

    def run_period(self):
        self.run_steps(self.period)
        return self.balance()

    def run(self, nsteps):
        """nsteps time steps with a balancer call after every full period."""
        end = self.t + nsteps
        while self.t < end:
            n = min(self.period, end - self.t)
            self.run_steps(n)
            if n == self.period:
                self.balance()
