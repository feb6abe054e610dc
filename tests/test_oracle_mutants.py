"""The oracle's pins against planted mistakes.

Each case copies the oracle, plants one plausible mistake in the copy (a
dropped term, a wrong sign, a wrong index or a transposed operand), and runs
every pin of test_oracle_pins.py (the step and its ctypes wrapper) or
test_balance_oracle.py (the balancers) against it. At least one pin must fail, so a mistake of that kind
in the oracle itself could not pass the pins unnoticed. Everything runs on
the CPU: the C step is compiled from a mutated copy of lb_oracle.c into a
temporary library, and the wrapper and the balancers are executed from
mutated copies of step.py and balance.py. An unmutated copy, built and run the same way, must pass every
pin; that guards against a harness fault being counted as a kill.

No mutant indexes outside its arrays: each either keeps its indexes in
range or goes through a range check of the original code.
"""
import importlib
import inspect
import itertools
import os
import subprocess

import pytest

from oracle import balance as B

import test_balance_oracle
import test_oracle_pins

ostep = importlib.import_module("oracle.step")   # the package's `step` is a function
ORACLE_DIR = os.path.dirname(os.path.abspath(ostep.__file__))
C_SRC = os.path.join(ORACLE_DIR, "lb_oracle.c")
PY_SRC = os.path.join(ORACLE_DIR, "balance.py")
WRAP_SRC = os.path.join(ORACLE_DIR, "step.py")

# (name, text in lb_oracle.c, replacement)
C_MUTANTS = [
    # advection (Sec. IV dynamics stand-in)
    ("adv_x_downwind", "long iu = i - sx;", "long iu = i + sx;"),
    ("adv_y_downwind", "long ju = j - sy;", "long ju = j + sy;"),
    ("adv_z_downwind", "long ku = k - sz;", "long ku = k + sz;"),
    ("adv_drops_y_term",
     "if (ay != 0.0) v += ay * (jin ? q[(k * ny + ju) * nx + i] : NAN);", ""),
    ("adv_cx_cy_transposed", "const double ax = fabs(g->cx), ay = fabs(g->cy)",
     "const double ax = fabs(g->cy), ay = fabs(g->cx)"),
    ("adv_signed_x_weight", "const double ax = fabs(g->cx)", "const double ax = g->cx"),
    ("adv_ignores_x_sign", "const long sx = g->cx >= 0 ? 1 : -1",
     "const long sx = 1"),
    ("adv_centre_weight_drops_cy", "double w0 = 1.0 - ax - ay - (down_open ? az : 0.0);",
     "double w0 = 1.0 - ax - (down_open ? az : 0.0);"),
    ("adv_closed_face_leaks", "double w0 = 1.0 - ax - ay - (down_open ? az : 0.0);",
     "double w0 = 1.0 - ax - ay - az;"),
    # the implicit solve (Fig. 1 / Fig. 4 column recurrence)
    ("thomas_first_row_interior", "double b0 = 1.0 + r * (nz > 1 ? 1.0 : 0.0);",
     "double b0 = 1.0 + r * (nz > 1 ? 2.0 : 0.0);"),
    ("thomas_last_row_interior", "double b = 1.0 + r * (k < nz - 1 ? 2.0 : 1.0);",
     "double b = 1.0 + r * 2.0;"),
    ("thomas_first_pivot_sign", "cp[0] = c0 / b0;", "cp[0] = -c0 / b0;"),
    ("thomas_pivot_drops_term", "double den = b - a * cp[k - 1];", "double den = b;"),
    ("thomas_pivot_sign", "double den = b - a * cp[k - 1];", "double den = b + a * cp[k - 1];"),
    ("thomas_forward_sign", "dp[k] = (d[k] - a * dp[k - 1]) / den;",
     "dp[k] = (d[k] + a * dp[k - 1]) / den;"),
    ("thomas_back_sign", "d[k] = dp[k] - cp[k] * d[k + 1];",
     "d[k] = dp[k] + cp[k] * d[k + 1];"),
    ("thomas_back_index", "d[k] = dp[k] - cp[k] * d[k + 1];",
     "d[k] = dp[k] - cp[k + 1] * d[k + 1];"),
    ("thomas_skips_row_0", "for (int32_t k = nz - 2; k >= 0; --k)",
     "for (int32_t k = nz - 2; k >= 1; --k)"),
    # k_c passes per column (Sec. VI-B load array)
    ("sweeps_one_extra", "for (int32_t s = 0; s < n; ++s)", "for (int32_t s = 0; s <= n; ++s)"),
    ("sweeps_skip_kc_1", "if (n <= 0) continue;", "if (n <= 1) continue;"),
    ("sweeps_kc_transposed", "int32_t n = kc[j * nx + i];", "int32_t n = kc[i * ny + j];"),
    ("sweeps_wrong_coefficient", "orc_thomas((int32_t)nz, g->r, col, cp, dp);",
     "orc_thomas((int32_t)nz, g->cx, col, cp, dp);"),
    # the moving-disk rule and the k_c array
    ("disk_strict_radius", "(dx * dx + dy * dy <= R * R)", "(dx * dx + dy * dy < R * R)"),
    ("disk_no_minimum_image_x", "if (dx > g->nx / 2) dx -= g->nx;", ""),
    ("disk_velocity_transposed",
     "long cxt = wrap((long)g->disk_x0 + t * (long)g->disk_vx, g->nx);",
     "long cxt = wrap((long)g->disk_x0 + t * (long)g->disk_vy, g->nx);"),
    ("kc_field_disk_transposed", "g->kc_mode ? orc_kc_disk(g, i, j, t)",
     "g->kc_mode ? orc_kc_disk(g, j, i, t)"),
    ("kc_field_array_transposed", ": g->kc[j * g->nx + i];", ": g->kc[i * g->ny + j];"),
    # compensated global sum
    ("sum_drops_compensation", "return s + c;", "return s;"),
    ("sum_branch_swapped", "if (fabs(s) >= fabs(v)) c += (s - t) + v;",
     "if (fabs(s) < fabs(v)) c += (s - t) + v;"),
    # runs over several steps, whole grid and window
    ("run_ignores_t0", "orc_kc_field(g, t0 + s, kc);", "orc_kc_field(g, s, kc);"),
    ("run_reuses_first_kc_array",
     "memcpy(kc, kc_fields + (size_t)s * ncol, sizeof(int32_t) * (size_t)ncol);",
     "memcpy(kc, kc_fields, sizeof(int32_t) * (size_t)ncol);"),
    ("window_disk_at_local_index",
     "orc_kc_disk(g, wrap(i0 + i, g->nx), wrap(j0 + j, g->ny), t0 + s)",
     "orc_kc_disk(g, i, j, t0 + s)"),
    ("window_kc_arrays_not_per_step",
     "kc_fields[(kc_per_step ? (size_t)s * ncol : 0) + j * wx + i]",
     "kc_fields[j * wx + i]"),
    # the weighted Jacobi sweep (Sec. IV "3D Jacobi solver" phase)
    ("jacobi_centre_weight", "w0 = 1.0 - 6.0 * g->nu;", "w0 = 1.0 - 5.0 * g->nu;"),
    ("jacobi_drops_j_plus", "sum += jpin ? q[(k * ny + jp) * nx + i] : NAN;", ""),
    ("jacobi_reflecting_top", "ku = k < nz - 1 ? k + 1 : nz - 1;",
     "ku = k < nz - 1 ? k + 1 : (nz > 1 ? nz - 2 : 0);"),
    ("jacobi_x_plus_is_self", "ip = wrap(ip, nx);", "ip = wrap(i, nx);"),
    ("dynamics_dispatch_inverted", "if (g->dynamics == 1) orc_jacobi",
     "if (g->dynamics != 1) orc_jacobi"),
]

# (name, text in step.py, replacement): the marshalling between numpy and C
WRAP_MUTANTS = [
    ("grid_disk_velocity_swapped", "kc, x0, y0, vx, vy, R,", "kc, x0, y0, vy, vx, R,"),
    ("grid_k_in_k_out_swapped", "self.k_in, self.k_out, self.dynamics, self.nu",
     "self.k_out, self.k_in, self.dynamics, self.nu"),
    ("window_x_wraps_by_ny", "ii = np.arange(i0, i0 + wx) % g.nx",
     "ii = np.arange(i0, i0 + wx) % g.ny"),
    ("run_drops_per_step_kc", "        kcp = kc_fields.ctypes.data\n", "        pass\n"),
]

# (name, text in balance.py, replacement)
PY_MUTANTS = [
    ("static_round_robin", "return [(v * nbins) // nvps for v in range(nvps)]",
     "return [v % nbins for v in range(nvps)]"),
    ("bin_loads_overwrites", "loads[b] += costs[v]", "loads[b] = costs[v]"),
    ("fixed_point_exponent_off_by_one", "e = 53 - n.bit_length() - x",
     "e = 54 - n.bit_length() - x"),
    ("fixed_point_truncates", "return [round(math.ldexp(c, e)) for c in costs]",
     "return [int(math.ldexp(c, e)) for c in costs]"),
    ("migrations_inverted", "zip(old, new) if a != b)", "zip(old, new) if a == b)"),
    ("greedy_lightest_first", "order = sorted(range(len(q)), key=lambda v: (-q[v], v))",
     "order = sorted(range(len(q)), key=lambda v: (q[v], v))"),
    ("greedy_ties_by_highest_id", "order = sorted(range(len(q)), key=lambda v: (-q[v], v))",
     "order = sorted(range(len(q)), key=lambda v: (-q[v], -v))"),
    ("blocked_heaviest_to_most_loaded",
     "bins = sorted(range(nbins), key=lambda b: (loads[b], b))",
     "bins = sorted(range(nbins), key=lambda b: (-loads[b], b))"),
    ("refine_threshold_below_mean", "thr = (1.0 + tol) * (float(sum(q)) / nbins)",
     "thr = (1.0 - tol) * (float(sum(q)) / nbins)"),
    ("refine_takes_least_loaded", "P = loads.index(lmax)", "P = loads.index(min(loads))"),
    ("refine_swap_bookkeeping_sign",
     "loads[P] -= d\n                loads[Q] += d",
     "loads[P] += d\n                loads[Q] -= d"),
]


def _mutate(src, before, after):
    assert src.count(before) == 1, "mutation site must occur exactly once: %r" % before
    return src.replace(before, after)


def _pin_cases(module):
    """Every test function of a pin module with every parameter set of its
    parametrize marks (cartesian product of stacked marks)."""
    cases = []
    for name, fn in sorted(vars(module).items(), key=lambda kv: _lineno(kv[1])):
        if not (name.startswith("test_") and callable(fn)):
            continue
        axes = []
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names, values = mark.args[0], mark.args[1]
            if isinstance(names, str):
                names = [s.strip() for s in names.split(",")]
            rows = [v if len(names) > 1 else (v,) for v in values]
            axes.append([dict(zip(names, row)) for row in rows])
        params = [{}] if not axes else [
            {k: v for d in combo for k, v in d.items()} for combo in itertools.product(*axes)]
        for kw in params:
            cases.append(("%s%s" % (name, kw if kw else ""), fn, kw))
    return cases


def _lineno(obj):
    try:
        return inspect.getsourcelines(obj)[1]
    except (TypeError, OSError):
        return 0


def _first_failing_pin(cases):
    """Name and error of the first pin that fails, or None if all pass."""
    for label, fn, kw in cases:
        try:
            fn(**kw)
        except Exception as e:           # an assertion, or a solve that broke down
            return label, "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")
    return None


def _build_c(src, path):
    with open(path + ".c", "w") as f:
        f.write(src)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", path, path + ".c", "-lm"])
    return path


def _use_c_library(monkeypatch, lib_path):
    """Point the oracle's ctypes wrapper at another build of the step."""
    monkeypatch.setattr(ostep, "_lib", None)
    monkeypatch.setattr(ostep, "build_oracle", lambda force=False: lib_path)


def _use_balance_source(monkeypatch, src):
    """Replace every function of oracle.balance with its definition in src."""
    ns = {"__name__": "oracle_balance_copy"}
    exec(compile(src, "balance_copy.py", "exec"), ns)
    for name, obj in vars(B).items():
        if inspect.isfunction(obj) and name in ns:
            monkeypatch.setattr(B, name, ns[name])


def _use_wrapper_source(monkeypatch, src):
    """Replace the oracle's public step functions (and the grid class the
    pins imported by name) by their definitions in src; the copy drives the
    unmutated C library."""
    ns = {"__name__": "oracle.step", "__file__": WRAP_SRC}
    exec(compile(src, "step_copy.py", "exec"), ns)
    import oracle
    for name in ("OracleGrid", "kc_field", "thomas", "advect", "jacobi", "step", "run",
                 "run_window", "compensated_sum"):
        monkeypatch.setattr(oracle, name, ns[name])
        if hasattr(test_oracle_pins, name):
            monkeypatch.setattr(test_oracle_pins, name, ns[name])


@pytest.fixture(scope="module")
def wrap_source():
    with open(WRAP_SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def c_source():
    with open(C_SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def py_source():
    with open(PY_SRC) as f:
        return f.read()


def test_unmutated_copies_pass_every_pin(c_source, wrap_source, py_source, tmp_path,
                                         monkeypatch):
    step_cases = _pin_cases(test_oracle_pins)
    bal_cases = _pin_cases(test_balance_oracle)
    assert len(step_cases) >= 40 and len(bal_cases) >= 100
    _use_c_library(monkeypatch, _build_c(c_source, str(tmp_path / "liborc_copy.so")))
    assert _first_failing_pin(step_cases) is None
    _use_wrapper_source(monkeypatch, wrap_source)
    assert _first_failing_pin(step_cases) is None
    _use_balance_source(monkeypatch, py_source)
    assert _first_failing_pin(bal_cases) is None


@pytest.mark.parametrize("name,before,after", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_step_pins_catch_planted_mistake(name, before, after, c_source, tmp_path, monkeypatch):
    lib = _build_c(_mutate(c_source, before, after), str(tmp_path / ("liborc_%s.so" % name)))
    _use_c_library(monkeypatch, lib)
    assert _first_failing_pin(_pin_cases(test_oracle_pins)) is not None, \
        "no pin fails with the mistake %r planted in the step oracle" % name


@pytest.mark.parametrize("name,before,after", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_balancer_pins_catch_planted_mistake(name, before, after, py_source, monkeypatch):
    _use_balance_source(monkeypatch, _mutate(py_source, before, after))
    assert _first_failing_pin(_pin_cases(test_balance_oracle)) is not None, \
        "no pin fails with the mistake %r planted in the balancer oracle" % name


@pytest.mark.parametrize("name,before,after", WRAP_MUTANTS, ids=[m[0] for m in WRAP_MUTANTS])
def test_wrapper_pins_catch_planted_mistake(name, before, after, wrap_source, monkeypatch):
    _use_wrapper_source(monkeypatch, _mutate(wrap_source, before, after))
    assert _first_failing_pin(_pin_cases(test_oracle_pins)) is not None, \
        "no pin fails with the mistake %r planted in the oracle's wrapper" % name
