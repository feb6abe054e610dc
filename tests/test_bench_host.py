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
