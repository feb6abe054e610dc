"""The C ABI library: loads, exports every entry point include/lb.h declares,
and its host balancers reproduce the oracle's assignments bit for bit.
No test here launches GPU work."""
import os
import random
import re

import numpy as np
import pytest

from oracle import balance as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbmod():
    from paper_1310_4218_gb300 import build
    build.build()
    from paper_1310_4218_gb300 import lb
    lb.load_library()
    return lb


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lbmod):
    names = declared_entry_points()
    assert len(names) >= 19
    lib = lbmod.load_library()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbmod.EXPORTED) == names


def test_plan_experiment_c(lbmod):
    costs = [2.0] * 8 + [1.0] * 8
    a, mig, pred = lbmod.lb_plan("greedy", costs, 4)
    assert mig == 12 and pred == 1.0
    assert list(a) == B.greedy(costs, 4)


@pytest.mark.parametrize("seed", range(25))
def test_plan_matches_oracle_bitwise(lbmod, seed):
    rng = random.Random(seed)
    nb = rng.randint(2, 40)
    nv = rng.randint(nb, 600)
    kind = seed % 3
    if kind == 0:
        costs = [rng.lognormvariate(0, 1) for _ in range(nv)]
    elif kind == 1:
        costs = [float(rng.randint(1, 5)) for _ in range(nv)]     # many ties
    else:
        costs = [rng.choice([1.0, 32.0]) * rng.uniform(0.9, 1.1) for _ in range(nv)]
    g, _, pg = lbmod.lb_plan("greedy", costs, nb)
    assert list(g) == B.greedy(costs, nb)
    assert pg == B.max_over_mean(costs, B.greedy(costs, nb), nb)
    cur = [rng.randrange(nb) for _ in range(nv)]
    r, mr, pr = lbmod.lb_plan("refine_swap", costs, nb, current=cur, refine_tol=0.05)
    ro = B.refine_swap(costs, cur, nb, 0.05)
    assert list(r) == ro
    assert mr == B.migrations(cur, ro)
    s, _, _ = lbmod.lb_plan("static", costs, nb)
    assert list(s) == B.static_blocks(nv, nb)


def test_plan_rejects_bad_input(lbmod):
    with pytest.raises(lbmod.LBError) as e:
        lbmod.lb_plan("greedy", [1.0, float("nan")], 2)
    assert e.value.status == lbmod.LB_EINVAL
    with pytest.raises(lbmod.LBError):
        lbmod.lb_plan("greedy", [1.0, -2.0], 2)
    with pytest.raises(lbmod.LBError):
        lbmod.lb_plan("queue", [1.0, 2.0], 2)
    for cur in ([0, 2], [-1, 0]):                # a present table outside [0, nprocs)
        with pytest.raises(lbmod.LBError) as e:
            lbmod.lb_plan("refine_swap", [1.0, 2.0], 2, current=cur)
        assert e.value.status == lbmod.LB_EINVAL and "current" in str(e.value)


def test_create_rejects_invalid_layout_before_touching_the_device(lbmod):
    """Validation runs first: an overlapping layout is refused with EINVAL."""
    g = lbmod.lb_grid_desc(8, 8, 4, 0.5, 0.5, 0.0, 0.1, lbmod.LB_F32, lbmod.LB_F32,
                           0x1000, 0x2000, None, 1, 0, 0, 0, 0, 1, 1, 1)
    vps = [(0, 0, 0, 8, 8), (0, 0, 0, 1, 1)]
    with pytest.raises(lbmod.LBError) as e:
        lbmod.lb_create([g], vps)
    assert e.value.status == lbmod.LB_EINVAL and "overlap" in str(e.value)
    with pytest.raises(lbmod.LBError) as e:
        lbmod.lb_create([g], [(0, 0, 0, 8, 7)])
    assert "gap" in str(e.value)
    bad = lbmod.lb_grid_desc(8, 8, 4, 0.7, 0.5, 0.0, 0.1, lbmod.LB_F32, lbmod.LB_F32,
                             0x1000, 0x2000, None, 1, 0, 0, 0, 0, 1, 1, 1)
    with pytest.raises(lbmod.LBError) as e:
        lbmod.lb_create([bad], [(0, 0, 0, 8, 8)])
    assert "cx" in str(e.value)


def test_create_validates_the_dynamics_fields_before_touching_the_device(lbmod):
    """dynamics is 0 (advection) or 1 (Jacobi); the Jacobi weight must lie in
    (0, 1/6]; a Jacobi grid ignores the Courant numbers; a row pitch is 0
    (dense) or at least nx, and pitch*ny*nz stays below 2^31."""
    def desc(cx, dynamics, nu, pad=0):
        return lbmod.lb_grid_desc(8, 8, 4, cx, 0.5, 0.0, 0.1, lbmod.LB_F32, lbmod.LB_F32,
                                  0x1000, 0x2000, None, 1, 0, 0, 0, 0, 1, 1, 1, dynamics, pad, nu)
    overlap = [(0, 0, 0, 8, 8), (0, 0, 0, 1, 1)]
    for d, word in ((desc(0.5, 2, 0.1), "dynamics"), (desc(0.5, 1, 0.0), "nu"),
                    (desc(0.5, 1, 0.2), "nu"), (desc(0.5, 1, -0.1), "nu"),
                    (desc(0.5, 0, 0.0, pad=1), "pitch"), (desc(0.5, 0, 0.0, pad=-8), "pitch"),
                    (desc(0.5, 0, 0.0, pad=1 << 27), "pitch*ny*nz")):
        with pytest.raises(lbmod.LBError) as e:
            lbmod.lb_create([d], overlap)
        assert e.value.status == lbmod.LB_EINVAL and word in str(e.value), str(e.value)
    # a valid Jacobi grid with out-of-range Courant numbers passes the grid
    # checks and fails only on the layout
    with pytest.raises(lbmod.LBError) as e:
        lbmod.lb_create([desc(5.0, 1, 1.0 / 7.0)], overlap)
    assert "overlap" in str(e.value)


def test_create_rejects_empty_inputs_and_sizes_out_of_range(lbmod):
    """No grid, no VP, zero or oversized extents, an FP64-compute column
    above 64 levels, mixed types or r across grids: each is refused with
    EINVAL before any device work."""
    def desc(nx=8, ny=8, nz=4, storage=lbmod.LB_F32, compute=lbmod.LB_F32, r=0.1, q0=0x1000):
        return lbmod.lb_grid_desc(nx, ny, nz, 0.5, 0.5, 0.0, r, storage, compute,
                                  q0, q0 + 0x1000, None, 1, 0, 0, 0, 0, 1, 1, 1)
    whole = [(0, 0, 0, 8, 8)]
    cases = [([], whole, "ngrids"), ([desc()], [], "VP"),
             ([desc(nx=0)], whole, "nx"), ([desc(ny=0)], whole, "nx"),
             ([desc(nz=0)], whole, "nz"), ([desc(nz=129)], whole, "nz"),
             ([desc(nx=2048, ny=2048, nz=512)], whole, "nz"),
             ([desc(nx=1 << 16, ny=1 << 16, nz=1)], whole, "2^31"),
             ([desc(nz=65, storage=lbmod.LB_F64, compute=lbmod.LB_F64)], whole, "nz <= 64"),
             ([desc(storage=lbmod.LB_BF16, compute=lbmod.LB_F64)], whole, "storage/compute"),
             ([desc(), desc(storage=lbmod.LB_F64, compute=lbmod.LB_F64, q0=0x9000)],
              whole + [(1, 0, 0, 8, 8)], "share storage"),
             ([desc(), desc(r=0.2, q0=0x9000)], whole + [(1, 0, 0, 8, 8)], "share r")]
    for grids, vps, word in cases:
        with pytest.raises(lbmod.LBError) as e:
            lbmod.lb_create(grids, vps)
        assert e.value.status == lbmod.LB_EINVAL and word in str(e.value), (word, str(e.value))
    with pytest.raises(lbmod.LBError) as e:
        lbmod.lb_plan("greedy", [], 4)
    assert e.value.status == lbmod.LB_EINVAL


@pytest.mark.parametrize("seed", range(10))
def test_plan_greedy_spatial_matches_oracle(lbmod, seed):
    rng = random.Random(500 + seed)
    nb = rng.randint(2, 30)
    nv = rng.randint(nb, 400)
    costs = [rng.lognormvariate(0, 1) for _ in range(nv)]
    g, _, _ = lbmod.lb_plan("greedy_spatial", costs, nb)
    assert list(g) == B.greedy_ordered(costs, nb, list(range(nv)))


@pytest.mark.parametrize("seed", range(10))
def test_plan_greedy_blocked_matches_oracle(lbmod, seed):
    rng = random.Random(700 + seed)
    nb = rng.randint(2, 30)
    nv = rng.randint(1, 400)
    costs = [rng.lognormvariate(0, 1) for _ in range(nv)]
    g, mig, pred = lbmod.lb_plan("greedy_blocked", costs, nb)
    ref = B.greedy_blocked(costs, nb, list(range(nv)))
    assert list(g) == ref
    assert pred == B.max_over_mean(costs, ref, nb)


@pytest.mark.parametrize("scale_exp", [-300, -20, 0, 20, 300])
@pytest.mark.parametrize("strategy", ["greedy", "greedy_blocked", "refine_swap"])
def test_plan_fixed_point_grid_at_any_cost_scale(lbmod, scale_exp, strategy):
    """The balancers' fixed-point grid (C++ llrint(ldexp)) equals the
    oracle's (Python round(ldexp)) for costs of any magnitude, zeros and
    exact ties included."""
    rng = random.Random(900 + scale_exp)
    nb = rng.randint(2, 40)
    nv = rng.randint(nb, 600)
    scale = 10.0 ** scale_exp
    costs = [rng.lognormvariate(0, 2) * scale for _ in range(nv)]
    for v in rng.sample(range(nv), nv // 10):
        costs[v] = 0.0
    for v in rng.sample(range(nv), nv // 10):
        costs[v] = costs[0]
    cur = [rng.randrange(nb) for _ in range(nv)]
    a, mig, pred = lbmod.lb_plan(strategy, costs, nb, current=cur)
    if strategy == "greedy":
        ref = B.greedy(costs, nb)
    elif strategy == "greedy_blocked":
        ref = B.greedy_blocked(costs, nb, list(range(nv)))
    else:
        ref = B.refine_swap(costs, cur, nb)
    assert list(a) == ref
    assert pred == B.max_over_mean(costs, ref, nb)
    assert mig == B.migrations(cur, ref)
