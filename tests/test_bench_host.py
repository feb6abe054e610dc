"""Host-side pieces of bench.py that need no GPU."""
import json
import sys

import numpy as np
import pytest

import bench


def line(sm, mx, reasons=("Not Active",) * 4):
    return "0, %d, %d, 500.0, 0x0, %s" % (sm, mx, ", ".join(reasons))


def test_clock_summary_keeps_the_timed_window_only():
    """Samples before the timed window (the idle lead-in) and after it do not
    count; the median comes from the samples under load."""
    stamped = [(0.0, line(2070, 2070)), (0.1, line(1200, 2070)), (0.2, line(1250, 2070)),
               (0.3, line(1300, 2070)), (0.5, line(2070, 2070))]
    c = bench.ClockSampler.summarise(stamped, (0.05, 0.35))
    assert c["sm_mhz"] == 1250 and c["samples"] == 3 and c["samples_in_timed_window"] == 3
    assert c["sm_max_mhz"] == 2070 and c["reasons"] == []


def test_clock_summary_reports_throttle_reasons():
    active = ("Not Active", "Active", "Not Active", "Active")
    stamped = [(1.0, line(1800, 2070, active)), (1.02, line(1810, 2070))]
    c = bench.ClockSampler.summarise(stamped, (0.9, 1.1))
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_short_window_falls_back_to_all_samples():
    """A window shorter than one sampling interval holds no sample: all are
    used, and the count inside is reported as 0."""
    stamped = [(0.0, line(2070, 2070)), (0.02, line(2060, 2070))]
    c = bench.ClockSampler.summarise(stamped, (0.005, 0.006))
    assert c["samples"] == 2 and c["samples_in_timed_window"] == 0
    assert bench.ClockSampler.summarise([], None)["sm_mhz"] is None


def args_for(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse()


CONTRACT_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                 "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    """--impl reference: W untimed oracle samples, then exactly K timed ones,
    bounded in total; one JSON line with the contract's keys, the oracle as
    its cpu_baseline and an e2e that moves no bytes."""
    budgets = []

    def fake_rate(w, budget_s=12.0):
        budgets.append(budget_s)
        return 2.0e8, "a patch", 5, 0.25

    monkeypatch.setattr(bench, "cpu_oracle_rate", fake_rate)
    args = args_for(monkeypatch, "--impl", "reference", "--steps", "4", "--warmup", "3")
    bench.run_reference(args, 0, 1)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert CONTRACT_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] == 2.0e8 and d["higher_is_better"] is True
    assert (d["steps"], d["warmup"], d["n_gpus"], d["ms_per_step"]) == (4, 3, 1, 250.0)
    assert d["config"]["workload"] == bench.DEFAULT_WORKLOAD
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": 2.0e8, "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert len(budgets) == 3 + 4
    assert sum(budgets) <= 60.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    def must_not_run(*a, **k):
        raise AssertionError("a rank other than 0 ran the oracle")

    monkeypatch.setattr(bench, "cpu_oracle_rate", must_not_run)
    args = args_for(monkeypatch, "--impl", "reference", "--gpus", "2")
    bench.run_reference(args, 1, 2)
    assert capsys.readouterr().out == ""


def test_cpu_oracle_sample_is_bounded_and_counts_its_patch():
    """The one-thread oracle sample stops after its budget, and its rate is
    the patch's nz * sum(k_c) per step over the time taken."""
    import oracle
    from workloads import get_config
    w = get_config("plain_fp64_64x64x32")
    v, desc, steps, dt = bench.cpu_oracle_rate(w, budget_s=0.3)
    assert steps >= 1 and 0.3 <= dt < 10.0
    g = w.grids[0]
    kc = oracle.kc_field(oracle.OracleGrid.from_spec(g), 0)     # the whole 64x64 grid
    assert v == pytest.approx(int(kc.sum(dtype=np.int64)) * g.nz * steps / dt, rel=1e-12)
    assert "64x64x32" in desc and "one thread" in desc


def test_traffic_figures_apply_only_to_the_sources_they_were_taken_on(tmp_path, monkeypatch):
    from paper_1310_4218_gb300.build import source_hash
    (tmp_path / "profiles").mkdir()
    entries = {"now": {"source_hash": source_hash(), "dram_bytes_per_step": 1.0},
               "before": {"source_hash": "0" * 16, "dram_bytes_per_step": 2.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entries))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("now") == entries["now"]
    assert bench.load_traffic("before") is None
    assert bench.load_traffic("absent") is None


def test_roofline_peak_prefers_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.roofline_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6674.5}))
    assert bench.roofline_peak() == (6674.5, "measured")


def test_whole_job_rate_on_one_rank():
    """Without a process group: this rank's work over its own time."""
    assert bench.whole_job_rate(3.0e9, 1500.0) == 2.0e9


def test_source_hash_ignores_comments_and_sees_code(tmp_path):
    """The hash that keys the recorded DRAM traffic survives comment-only
    edits and changes with any code edit; literals that contain comment
    markers are code."""
    import shutil
    from paper_1310_4218_gb300 import build
    csrc, inc = tmp_path / "csrc", tmp_path / "include"
    shutil.copytree(build.CSRC, csrc)
    shutil.copytree(build.INCLUDE, inc)
    h0 = build.source_hash(str(csrc), str(inc))
    assert h0 == build.source_hash()
    f = csrc / "lb_step_f32.cu"
    text = f.read_text()
    f.write_text("// a new comment\n/* and a block\n   comment */\n" + text + "\n\n")
    assert build.source_hash(str(csrc), str(inc)) == h0
    f.write_text(text + "\nstatic const int lb_unused_constant = 1;\n")
    assert build.source_hash(str(csrc), str(inc)) != h0
    assert build.strip_comments('a = "//x"; // c\nb = \'/\'; /* d */ c;\n') == \
        'a = "//x";\nb = \'/\';   c;'


class _FakeLB:
    """Records the calls StrategyRun makes; no library, no GPU."""
    LB_ATOMIC_QUEUE = 3

    def __init__(self):
        self.kc_installs = []
        self.rows = 0

    def lb_set_kc(self, ctx, grid, ptr):
        self.kc_installs.append((grid, ptr))

    def lb_device_measure(self, ctx):
        pass

    def lb_device_rebalance_if(self, ctx, strategy, threshold):
        self.rows += 1

    def lb_graph_create_periods(self, ctx, nsteps, strategy, measure, threshold):
        return object()

    def lb_graph_launch(self, ctx, gexec):
        self.rows += 1

    def lb_balance_history(self, ctx):
        return [[0, 7, 0, 1.0, 1.05, 1.0, 0, 0]] * self.rows


class _FakeSim:
    ctx = None

    def __init__(self):
        self.steps = []

    def step(self, n):
        self.steps.append(n)


class _Arr:
    def __init__(self, e):
        self.e = e

    def data_ptr(self):
        return 1000 + self.e


def _fake_run(strategy, period, epoch_steps, epochs):
    run = object.__new__(bench.StrategyRun)
    parts = strategy.split("+")
    flags = set(parts[1:])
    run.lb, run.sim = _FakeLB(), _FakeSim()
    run.w = type("W", (), {"kc_epoch_steps": epoch_steps, "grids": [None]})()
    run.epochs = epochs
    run.kc_dev = {e: [_Arr(e)] for e in epochs}
    run.dev_mode = "dev" in flags
    run.predict = "pred" in flags and run.dev_mode
    run.threshold = "thr" in flags and run.dev_mode
    run.use_graph = "graph" in flags and run.dev_mode
    run.gexec, run.kc_epoch, run.dev_tags, run.kernels = None, None, [], 0
    run.P, run.strategy, run.t, run.stats, run.timed_rows = period, parts[0], 0, {}, []
    run.name = strategy
    run.info = type("Info", (), {"strategy": 3 if parts[0] == "queue" else 7})()
    return run


@pytest.mark.parametrize("steps,warmup", [(20, 5), (40, 3), (5, 5), (1, 3), (7, 4), (15, 0)])
@pytest.mark.parametrize("strategy", ["greedy_blocked+steal+dev+pred+thr",
                                      "greedy_blocked+steal+dev+pred+thr+graph",
                                      "greedy_blocked+dev", "queue+dev"])
def test_every_k_c_epoch_the_run_asks_for_is_drawn(monkeypatch, steps, warmup, strategy):
    """The bench's period loop over warm-up, timed and end-to-end periods
    (the headline ctx runs its share of the end-to-end ring) only installs
    k_c arrays of epochs that were drawn, for any (steps, warmup); each
    time step runs under the epoch of its index, and the balancer call
    after a period may install the next period's array."""
    args = args_for(monkeypatch, "--steps", str(steps), "--warmup", str(warmup))
    epoch_steps, P = 50, args.period
    total = bench.total_time_steps(args)
    epochs = {e: None for e in bench.epochs_needed(total, epoch_steps)}
    shares = [(args.steps + bench.E2E_RING - 1 - x) // bench.E2E_RING
              for x in range(bench.E2E_RING)]
    assert sum(shares) == args.steps
    for x, share in enumerate(shares):
        run = _fake_run(strategy, P, epoch_steps, epochs)
        nper = warmup + (steps if x == 0 else 0) + share
        for _ in range(nper):
            run.launches(run.t, run.t + P)
            run.balance("p", run.t + P)
            run.t += P
        assert run.kc_epoch in epochs
        if not run.use_graph:
            assert sum(run.sim.steps) == nper * P


def test_epochs_cover_the_step_after_the_last():
    assert list(bench.epochs_needed(450, 50)) == list(range(10))
    assert list(bench.epochs_needed(449, 50)) == list(range(9))
    assert list(bench.epochs_needed(0, 50)) == [0]
    assert list(bench.epochs_needed(100, 0)) == []


def test_reference_arm_names_the_same_workload_config(monkeypatch, capsys):
    """Both arms print the same config object for the same arguments."""
    monkeypatch.setattr(bench, "cpu_oracle_rate", lambda w, budget_s=12.0: (1.0, "p", 1, 0.1))
    args = args_for(monkeypatch, "--impl", "reference", "--steps", "1", "--warmup", "0")
    bench.run_reference(args, 0, 1)
    d = json.loads(capsys.readouterr().out)
    from workloads import get_config
    assert d["config"] == bench.bench_config(get_config(args.workload), args, 1)
