"""Device-side measurement and rebalancing (Sec. V, VI on the GPU): for equal
costs and current assignment the device balancers give the host balancers'
(and the oracle's) assignments, migrations and predicted max/mean bit for
bit; their tables drive steps with unchanged values; a graph of whole
rebalance periods replays like direct steps."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import balance as B  # noqa: E402
from gpu_common import Grid, item_kc, normwise, random_field, round_to_storage  # noqa: E402
from workloads import regular_blocks  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def make_sim(grids, fields, vps, **opt):
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    o = lb.lb_default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return Simulation(grids, fields, vps, options=o)


def spatial_order(vps):
    return sorted(range(len(vps)), key=lambda v: (vps[v][0], vps[v][2], vps[v][1], v))


def costs_of(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.uniform(1.0, 100.0, n)
    if kind == "ties":                     # many equal costs: tie-breaking
        return rng.integers(1, 5, n).astype(np.float64)
    if kind == "heavy":                    # a few heavy VPs: swaps
        c = rng.uniform(0.9, 1.1, n)
        idx = rng.choice(n, max(1, n // 30), replace=False)
        c[idx] = rng.uniform(50.0, 200.0, idx.size)
        return c
    if kind == "zeros":                    # zero-cost VPs are never moved alone
        c = rng.uniform(0.0, 10.0, n)
        c[rng.random(n) < 0.3] = 0.0
        return c
    raise ValueError(kind)


LAYOUTS = {
    # name: (nx, ny, vp_w, vp_h)
    "64vps": (64, 32, 8, 4),
    "1536vps": (128, 96, 4, 2),
    "4800vps": (160, 120, 2, 2),
}


def small_grid(nx, ny, nz=8, prec="f32"):
    return Grid(nx, ny, nz, storage=prec, compute=prec, disk=(5, 7, 1, 1, 6), k_in=5, k_out=1)


def twin(layout, nz=8, prec="f32", **opt):
    nx, ny, w, h = LAYOUTS[layout]
    g = small_grid(nx, ny, nz, prec)
    q = round_to_storage(random_field(g, 3), prec)
    vps = regular_blocks(nx, ny, w, h)
    return g, q, vps, make_sim([g], [q], vps, **opt), make_sim([g], [q], vps, **opt)


def hist_last(ctx):
    from paper_1310_4218_gb300 import lb
    return lb.lb_balance_history(ctx)[-1]


@pytest.mark.parametrize("layout", list(LAYOUTS))
@pytest.mark.parametrize("kind", ["uniform", "ties", "heavy", "zeros"])
@pytest.mark.parametrize("strategy", ["greedy", "greedy_spatial", "greedy_blocked", "refine_swap",
                                      "static"])
def test_device_balancer_equals_host(layout, kind, strategy):
    from paper_1310_4218_gb300 import lb
    g, q, vps, dev, host = twin(layout)
    nv = len(vps)
    nb = dev.info().nprocs
    rng = np.random.default_rng(7)
    cur = rng.integers(0, nb, nv).astype(np.int32)      # a scrambled current table
    costs = costs_of(kind, nv, 11)
    for s in (dev, host):
        s.set_costs(costs)
        lb.lb_set_assignment(s.ctx, cur)
    lb.lb_device_rebalance(dev.ctx, strategy)
    a_dev, _ = dev.assignment()
    mig_h, pred_h = host.rebalance(strategy)
    a_host, _ = host.assignment()
    row = hist_last(dev.ctx)
    dev.close()
    host.close()
    assert np.array_equal(a_dev, a_host)
    # the oracle's assignment and predicted max/mean, independently
    c = list(map(float, costs))
    if strategy == "greedy":
        ref = B.greedy(c, nb)
    elif strategy == "greedy_spatial":
        ref = B.greedy_ordered(c, nb, spatial_order(vps))
    elif strategy == "greedy_blocked":
        ref = B.greedy_blocked(c, nb, spatial_order(vps))
    elif strategy == "refine_swap":
        ref = B.refine_swap(c, list(map(int, cur)), nb, tol=0.05)
    else:
        ref = B.static_blocks(nv, nb)
    assert list(a_dev) == ref
    assert row[1] == lb.STRATEGIES[strategy]
    assert row[2] == mig_h == B.migrations(list(map(int, cur)), ref)
    assert row[3] == pred_h == B.max_over_mean(c, ref, nb)


def test_auto_strategies_switch_on_the_device():
    """LB_AUTO_SPATIAL: list scheduling on the first device rebalance, then
    RefineSwapLB from the table it made -- like the host path."""
    from paper_1310_4218_gb300 import lb
    g, q, vps, dev, host = twin("1536vps")
    nv = len(vps)
    for k, seed in enumerate((1, 2, 3)):
        costs = costs_of("heavy" if k else "uniform", nv, seed)
        dev.set_costs(costs)
        host.set_costs(costs)
        lb.lb_device_rebalance(dev.ctx, "auto_spatial")
        host.rebalance("auto_spatial")
        assert np.array_equal(dev.assignment()[0], host.assignment()[0])
    rows = lb.lb_balance_history(dev.ctx)
    assert list(rows[:, 1]) == [lb.LB_GREEDY_SPATIAL, lb.LB_REFINE_SWAP, lb.LB_REFINE_SWAP]
    # the host balancer continues from the device's table
    costs = costs_of("ties", nv, 4)
    dev.set_costs(costs)
    cur = dev.assignment()[0]
    dev.rebalance("refine_swap")
    ref, _, _ = lb.lb_plan("refine_swap", costs, dev.info().nprocs, current=cur)
    assert np.array_equal(dev.assignment()[0], ref)
    dev.close()
    host.close()


@pytest.mark.parametrize("ctas", [2, 4])
def test_more_processors_than_the_register_greedy(ctas):
    """Two or four processors per SM (304 or 608 processors, over 256: the
    nz-96 FP32 kernels for shared SMs): GreedyLB keeps its loads in shared
    memory instead of registers."""
    from paper_1310_4218_gb300 import lb
    g, q, vps, dev, host = twin("4800vps", nz=96, prec="f32", ctas_per_sm=ctas)
    nb = dev.info().nprocs
    assert nb == ctas * dev.info().nsm and nb > 256
    costs = costs_of("ties", len(vps), 5)
    for strategy in ("greedy", "greedy_spatial", "greedy_blocked", "refine_swap"):
        dev.set_costs(costs)
        host.set_costs(costs)
        lb.lb_device_rebalance(dev.ctx, strategy)
        host.rebalance(strategy)
        assert np.array_equal(dev.assignment()[0], host.assignment()[0]), strategy
        costs = costs_of("heavy", len(vps), 6)
    dev.close()
    host.close()


def test_device_measurement_is_the_host_cost_average():
    """lb_device_measure folds cycles into the cost average with the host's
    FP64 formula: the first measurement is the average, later ones
    a*last + (1-a)*previous, bit for bit; costs follow the sweep count."""
    from paper_1310_4218_gb300 import lb
    g = Grid(256, 256, 64, disk=(64, 64, 0, 0, 40), k_in=32, k_out=1)
    q = round_to_storage(random_field(g, 15), "f32")
    vps = regular_blocks(256, 256, 32, 32)
    sim = make_sim([g], [q], vps)
    sim.step(3)
    lb.lb_device_measure(sim.ctx)
    avg1, last1 = lb.lb_get_costs(sim.ctx, len(vps))
    sim.step(2)
    lb.lb_device_measure(sim.ctx)
    avg2, last2 = lb.lb_get_costs(sim.ctx, len(vps))
    assert np.all(last1 > 0) and np.all(last2 > 0)
    assert np.array_equal(avg1, last1)
    a = 0.5
    assert np.array_equal(avg2, np.float64(a) * last2 + np.float64(1.0 - a) * avg1)
    # heavier VPs (the disk) cost more
    kc = oracle.kc_field(g.oracle(), 0)
    sweeps = np.array([kc[y0:y0 + h, x0:x0 + w].sum() for (_, x0, y0, w, h) in vps], float)
    assert np.corrcoef(sweeps, last2)[0, 1] > 0.8
    # no step since the last measurement: reported at the next sync
    lb.lb_device_measure(sim.ctx)
    with pytest.raises(lb.LBError) as ei:
        lb.lb_sync(sim.ctx)
    assert ei.value.status == lb.LB_ESTATE
    # the host measurement sees the device's state and carries on from it
    sim.step(1)
    cost, _ = sim.measure()
    avg3, _ = lb.lb_get_costs(sim.ctx, len(vps))
    assert np.array_equal(avg3, np.float64(a) * cost + np.float64(1.0 - a) * avg2)
    sim.close()


def test_device_tables_drive_steps_with_unchanged_values():
    """Steps under device-made tables (with and without stealing) give the
    bits of a static run and the oracle's values; the work counter agrees."""
    from paper_1310_4218_gb300 import lb
    g = Grid(96, 80, 32, disk=(20, 30, 1, 1, 14), k_in=24, k_out=1)
    q = round_to_storage(random_field(g, 33), "f32")
    vps = regular_blocks(96, 80, 8, 8)
    base = make_sim([g], [q], vps)
    base.step(12)
    ref_bits = base.field(0)
    w_base = lb.lb_work_done(base.ctx)
    base.close()
    for steal in (0, 1):
        sim = make_sim([g], [q], vps, steal=steal)
        for strategy in ("greedy", "refine_swap", "greedy_spatial", "greedy_blocked"):
            sim.step(3)
            lb.lb_device_measure(sim.ctx)
            lb.lb_device_rebalance(sim.ctx, strategy)
        out = sim.field(0)
        assert lb.lb_work_done(sim.ctx) == w_base
        a, nb = sim.assignment()
        assert a.min() >= 0 and a.max() < nb
        sim.close()
        assert np.array_equal(out, ref_bits)
    ref, _ = oracle.run(g.oracle(), q, 12)
    assert normwise(ref_bits, ref) <= 1e-5


def test_graph_of_rebalance_periods():
    """One graph of 3 periods (2 steps, device measurement, device
    rebalance), replayed twice: the bits of 12 direct steps, 6 history rows
    (list scheduling, then RefineSwapLB), step counters advanced."""
    from paper_1310_4218_gb300 import lb
    g = Grid(80, 48, 32, disk=(10, 40, 1, 2, 9), k_in=11, k_out=1)
    q = round_to_storage(random_field(g, 41), "f32")
    vps = regular_blocks(80, 48, 8, 4)
    a = make_sim([g], [q], vps)
    a.step(12)
    ref = a.field(0)
    a.close()
    b = make_sim([g], [q], vps, steal=1)
    graph = lb.lb_graph_create_periods(b.ctx, 2, "auto_spatial", 3, 0.0)
    lb.lb_graph_launch(b.ctx, graph)
    lb.lb_graph_launch(b.ctx, graph)
    out = b.field(0)
    rows = lb.lb_balance_history(b.ctx)
    info = b.info()
    assign, nb = b.assignment()
    lb.lb_graph_destroy(b.ctx, graph)
    b.close()
    assert np.array_equal(out, ref)
    assert info.step == 12
    assert len(rows) == 6
    assert list(rows[:, 0]) == [2, 4, 6, 8, 10, 12]
    assert list(rows[:, 1]) == [lb.LB_GREEDY_SPATIAL] + [lb.LB_REFINE_SWAP] * 5
    assert np.all(rows[:, 3] >= 0.99) and np.all(rows[:, 4] >= 0.99)
    assert assign.min() >= 0 and assign.max() < nb


def test_device_balancer_refusals():
    from paper_1310_4218_gb300 import lb
    g = small_grid(64, 32)
    q = round_to_storage(random_field(g, 1), "f32")
    vps = regular_blocks(64, 32, 8, 4)
    sim = make_sim([g], [q], vps)
    # no costs yet: reported at the next sync, table unchanged
    before = sim.assignment()[0]
    lb.lb_device_rebalance(sim.ctx, "greedy")
    with pytest.raises(lb.LBError) as ei:
        lb.lb_sync(sim.ctx)
    assert ei.value.status == lb.LB_ESTATE
    assert np.array_equal(sim.assignment()[0], before)
    with pytest.raises(lb.LBError) as ei:
        lb.lb_device_rebalance(sim.ctx, "queue")
    assert ei.value.status == lb.LB_ESTATE
    sim.step(1)
    sim.measure()
    sim.rebalance("queue")
    with pytest.raises(lb.LBError) as ei:
        lb.lb_device_rebalance(sim.ctx, "greedy")
    assert ei.value.status == lb.LB_ESTATE
    # queue mode: device measurement and a record of the period, no table
    before = sim.assignment()[0]
    sim.step(2)
    lb.lb_device_measure(sim.ctx)
    lb.lb_device_rebalance(sim.ctx, "queue")
    row = lb.lb_balance_history(sim.ctx)[-1]
    assert row[1] == lb.LB_ATOMIC_QUEUE and row[2] == 0 and row[3] == row[5] >= 1.0
    assert np.array_equal(sim.assignment()[0], before)
    assert sim.info().strategy == lb.LB_ATOMIC_QUEUE
    sim.close()
    # more VPs than the device balancer takes
    g2 = Grid(2, 4097, 4, disk=(0, 0, 0, 0, 1), k_in=1, k_out=1)
    q2 = round_to_storage(random_field(g2, 2), "f32")
    big = make_sim([g2], [q2], regular_blocks(2, 4097, 1, 1))
    with pytest.raises(lb.LBError) as ei:
        lb.lb_device_measure(big.ctx)
    assert ei.value.status == lb.LB_EINVAL
    big.close()


def test_schedule_in_device_mode():
    """Schedule(device=True): periods of steps, device measurement and device
    rebalancing with a k_c array re-drawn between segments; the values are
    the oracle's and one history row is kept per period."""
    from paper_1310_4218_gb300.schedule import Schedule
    from workloads.kcfield import lognormal_kc
    g = Grid(96, 64, 32, kc_disk=False)
    q = round_to_storage(random_field(g, 61), "f32")
    vps = regular_blocks(96, 64, 8, 8)
    kcs = {e: [lognormal_kc(96, 64, 99, e)] for e in range(3)}
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    sim = Simulation([g], [q], vps, kc_arrays=kcs[0], options=lb.lb_default_options())
    sch = Schedule(sim, 4, "auto_spatial", kc_epochs=kcs, epoch_steps=5, device=True)
    sch.run(12)
    hist = sch.device_history()
    out = sim.field(0)
    sim.close()
    assert [h["step"] for h in hist] == [4, 8, 12]
    assert [h["strategy"] for h in hist] == [lb.LB_GREEDY_SPATIAL, lb.LB_REFINE_SWAP,
                                             lb.LB_REFINE_SWAP]
    kc_of = lambda t: kcs[t // 5][0]
    ref = q
    for t in range(12):
        ref, _ = oracle.run(g.oracle(kc_of(t)), ref, 1, t0=t)
    assert normwise(out, ref) <= 1e-5


def test_kc_redraw_rescales_costs_by_the_fitted_model():
    """lb_set_kc with predict_kc: every cost average is multiplied by
    (kappa f1 + f2_new) / (kappa f1 + f2_old), f1 = items * nz, f2 = nz *
    sum over items of the largest k_c, kappa from the least-squares fit of
    the last measured costs to (f1, f2_old).  Checked against a numpy
    restatement (FP64; the device sums in another order, hence rtol)."""
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    from workloads.kcfield import lognormal_kc
    g = Grid(96, 64, 32, kc_disk=False)
    q = round_to_storage(random_field(g, 81), "f32")
    vps = regular_blocks(96, 64, 8, 8)
    kc0 = lognormal_kc(96, 64, 5, 0)
    kc1 = lognormal_kc(96, 64, 5, 1)
    o = lb.lb_default_options()
    o.predict_kc = 1
    sim = Simulation([g], [q], vps, kc_arrays=[kc0], options=o)
    nv = len(vps)
    sim.step(4)
    lb.lb_device_measure(sim.ctx)
    avg0, last0 = lb.lb_get_costs(sim.ctx, nv)
    sim.set_kc(0, kc1)
    avg1, _ = lb.lb_get_costs(sim.ctx, nv)
    info = sim.info()
    sim.step(2)
    out = sim.field(0)
    sim.close()

    def feats(kc):
        f1, f2 = [], []
        for vp in vps:
            chunks = item_kc(np.maximum(kc, 0), vp, info.item_w, info.item_h)
            f1.append(len(chunks) * g.nz)
            f2.append(sum(int(c.max()) for c in chunks) * g.nz)
        return np.array(f1, float), np.array(f2, float)
    assert sum(len(item_kc(kc0, vp, info.item_w, info.item_h)) for vp in vps) == info.work_items
    f1, f2o = feats(kc0)
    _, f2n = feats(kc1)
    a11, a12, a22 = (f1 * f1).sum(), (f1 * f2o).sum(), (f2o * f2o).sum()
    b1, b2 = (f1 * last0).sum(), (f2o * last0).sum()
    det = a11 * a22 - a12 * a12
    kappa = 6.0
    if det > 1e-9 * a11 * a22 and a22 > 0:
        a, b = (b1 * a22 - b2 * a12) / det, (a11 * b2 - a12 * b1) / det
        if b > 0 and a >= 0:
            kappa = a / b
    expect = avg0 * ((kappa * f1 + f2n) / (kappa * f1 + f2o))
    assert np.allclose(avg1, expect, rtol=1e-9, atol=0.0)
    assert not np.allclose(avg1, avg0)
    # values are unaffected by the cost model
    ref, _ = oracle.run(g.oracle(kc0), q, 4)
    ref, _ = oracle.run(g.oracle(kc1), ref, 2, t0=4)
    assert normwise(out, ref) <= 1e-5


def test_device_threshold_keeps_a_good_table():
    """lb_device_rebalance_if keeps the table while its predicted max/mean
    under the current costs is within the threshold, rebalances (exactly as
    the host balancer) once it is not, and is forced to rebalance after a
    k_c rescale; steps under kept tables keep their values."""
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    from workloads.kcfield import lognormal_kc
    g = Grid(96, 64, 32, kc_disk=False)
    q = round_to_storage(random_field(g, 91), "f32")
    vps = regular_blocks(96, 64, 4, 4)
    kc0 = lognormal_kc(96, 64, 8, 0)
    kc1 = lognormal_kc(96, 64, 8, 1)
    o = lb.lb_default_options()
    o.predict_kc = 1
    sim = Simulation([g], [q], vps, kc_arrays=[kc0], options=o)
    nv, nb = len(vps), sim.info().nprocs
    c1 = costs_of("uniform", nv, 3)
    sim.set_costs(c1)
    lb.lb_device_rebalance(sim.ctx, "greedy_blocked")
    t1 = sim.assignment()[0]
    # 2-3 VPs per processor: the table just made predicts well below 3
    lb.lb_device_rebalance_if(sim.ctx, "greedy_blocked", 3.0)      # good enough: kept
    row = lb.lb_balance_history(sim.ctx)[-1]
    assert row[7] == 1 and row[2] == 0 and row[3] <= 3.0
    assert np.array_equal(sim.assignment()[0], t1)
    sim.step(2)
    c2 = costs_of("heavy", nv, 4)
    sim.set_costs(c2)
    lb.lb_device_rebalance_if(sim.ctx, "greedy_blocked", 1.01)     # unbalanced: rebalanced
    row = lb.lb_balance_history(sim.ctx)[-1]
    ref = B.greedy_blocked(list(map(float, c2)), nb, spatial_order(vps))
    assert row[7] == 0 and list(sim.assignment()[0]) == ref
    sim.step(2)
    lb.lb_device_measure(sim.ctx)
    sim.set_kc(0, kc1)                                             # rescale forces
    lb.lb_device_rebalance_if(sim.ctx, "greedy_blocked", 1e9)
    row = lb.lb_balance_history(sim.ctx)[-1]
    assert row[7] == 0
    lb.lb_device_rebalance_if(sim.ctx, "greedy_blocked", 1e9)      # then kept again
    assert lb.lb_balance_history(sim.ctx)[-1][7] == 1
    sim.step(3)
    out = sim.field(0)
    sim.close()
    ref, _ = oracle.run(g.oracle(kc0), q, 4)
    ref, _ = oracle.run(g.oracle(kc1), ref, 3, t0=4)
    assert normwise(out, ref) <= 1e-5


def test_autotuner_picks_the_fastest_candidate_and_caches(tmp_path):
    from paper_1310_4218_gb300.autotune import autotune
    g = Grid(128, 96, 32, disk=(30, 30, 1, 1, 20), k_in=24, k_out=1)
    q = round_to_storage(random_field(g, 5), "f32")
    vps = regular_blocks(128, 96, 16, 16)
    cache = str(tmp_path / "tune.json")
    res = autotune([g], [q], vps, cache=cache, strategies=("greedy_blocked", "queue"),
                   periods=(4,), variants=(0,), splits=(1, 2))
    vals = [c["value"] for c in res["candidates"] if c["value"]]
    assert len(res["candidates"]) == 4 and len(vals) == 4
    assert res["value"] == max(vals)
    again = autotune([g], [q], vps, cache=cache, strategies=("greedy_blocked", "queue"),
                     periods=(4,), variants=(0,), splits=(1, 2))
    assert again == res
