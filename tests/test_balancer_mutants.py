"""The host balancer's parity tests against planted mistakes.

The library's host balancers (csrc/lb_balance.cpp, reached through
lb_plan) are held bit for bit to the oracle's by the lb_plan tests of
test_abi.py.  Each case here plants one plausible mistake in a copy of
lb_balance.cpp, compiles that copy with the library's own flags, links it
with the library's other objects into a temporary liblb.so, and runs every
lb_plan test against it.  At least one must fail.  An unmutated copy,
built the same way, must pass them all.  Host code only: nothing here
touches a GPU.

No mutant indexes outside its arrays: every bin index it produces stays
in [0, nbins).
"""
import os
import subprocess

import pytest

import test_abi
from test_oracle_mutants import _first_failing_pin, _mutate, _pin_cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in lb_balance.cpp, replacement)
MUTANTS = [
    ("static_round_robin", "out[v] = (int)(((long long)v * nbins) / nvps);",
     "out[v] = v % nbins;"),
    ("fixed_point_truncates", "q[v] = std::llrint(std::ldexp(costs[v], e));",
     "q[v] = (long long)(std::ldexp(costs[v], e));"),
    ("fixed_point_exponent_off_by_one", "const int e = 53 - bit_length((long long)n) - x;",
     "const int e = 52 - bit_length((long long)n) - x;"),
    ("mean_over_objects", "const double mean = (double)total / (double)nbins;",
     "const double mean = (double)total / (double)q.size();"),
    ("migrations_inverted", "m += a[v] != b[v];", "m += a[v] == b[v];"),
    ("list_schedule_most_loaded", "std::vector<Item>, std::greater<Item>>",
     "std::vector<Item>, std::less<Item>>"),
    ("greedy_lightest_first",
     "std::sort(order.begin(), order.end(), [&](int a, int b) {\n"
     "        if (q[a] != q[b]) return q[a] > q[b];",
     "std::sort(order.begin(), order.end(), [&](int a, int b) {\n"
     "        if (q[a] != q[b]) return q[a] < q[b];"),
    ("greedy_ties_by_highest_id",
     "        return a < b;\n    });\n    list_schedule(q, nbins, order, out);",
     "        return a > b;\n    });\n    list_schedule(q, nbins, order, out);"),
    ("blocked_heaviest_to_most_loaded",
     "            if (loads[a] != loads[b]) return loads[a] < loads[b];\n"
     "            return a < b;\n        });\n        for (size_t k",
     "            if (loads[a] != loads[b]) return loads[a] > loads[b];\n"
     "            return a < b;\n        });\n        for (size_t k"),
    ("refine_threshold_below_mean", "const double thr = (1.0 + tol) *",
     "const double thr = (1.0 - tol) *"),
    ("refine_takes_least_loaded", "if (loads[b] > loads[P]) P = b;",
     "if (loads[b] < loads[P]) P = b;"),
    ("refine_move_tests_the_source", "(double)(loads[Q] + q[o]) <= thr",
     "(double)(loads[P] + q[o]) <= thr"),
    ("refine_swap_bookkeeping_sign",
     "                loads[P] -= d;\n                loads[Q] += d;",
     "                loads[P] += d;\n                loads[Q] -= d;"),
]


@pytest.fixture(scope="module")
def parts():
    """The library's objects (built if stale), the balancer's source and the
    plan tests to run."""
    from paper_1310_4218_gb300 import build
    build.build()
    objs = sorted(os.path.join(build.BUILD, f) for f in os.listdir(build.BUILD)
                  if f.endswith(".o") and f != "lb_balance.cpp.o")
    with open(os.path.join(build.CSRC, "lb_balance.cpp")) as f:
        src = f.read()
    cases = [c for c in _pin_cases(test_abi) if c[0].startswith("test_plan")]
    assert len(cases) >= 40
    return build, objs, src, cases


def _build_variant(build, objs, src, out_dir, tag):
    cpp = os.path.join(out_dir, "lb_balance_%s.cpp" % tag)
    obj = cpp + ".o"
    lib = os.path.join(out_dir, "liblb_%s.so" % tag)
    with open(cpp, "w") as f:
        f.write(src)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I",
                           build.INCLUDE, "-I", build.CSRC, "-I", "/usr/local/cuda/include",
                           "-c", cpp, "-o", obj])
    subprocess.check_call([build._nvcc()] + build.ARCH + ["-shared", "-cudart", "static",
                                                          "-o", lib] + objs + [obj])
    return lib


def _run_plan_tests(monkeypatch, lib_path, cases):
    from paper_1310_4218_gb300 import lb
    monkeypatch.setattr(lb, "_lib", None)
    lb.load_library(lib_path)
    return _first_failing_pin([(label, fn, dict(kw, lbmod=lb)) for label, fn, kw in cases])


def test_unmutated_copy_passes_every_plan_test(parts, tmp_path, monkeypatch):
    build, objs, src, cases = parts
    lib = _build_variant(build, objs, src, str(tmp_path), "copy")
    assert _run_plan_tests(monkeypatch, lib, cases) is None


@pytest.mark.parametrize("name,before,after", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_plan_tests_catch_planted_mistake(name, before, after, parts, tmp_path, monkeypatch):
    build, objs, src, cases = parts
    lib = _build_variant(build, objs, _mutate(src, before, after), str(tmp_path), name)
    assert _run_plan_tests(monkeypatch, lib, cases) is not None, \
        "no lb_plan test fails with the mistake %r planted in the host balancer" % name
