"""The dataflow step kernel (lb_options.dataflow with the atomic queue): a
launch's steps without a grid barrier, each work item waiting only for the
items that own its columns' neighbours.  Its fields must equal the barrier
kernel's bit for bit (same arithmetic per column) and the oracle's, its
global sums the barrier run's to FP64 rounding, on either upwind side, with
the Jacobi sweep (which reads both sides), over launches of many steps,
under CUDA-graph replay; a 1 ns wait limit must end a launch with
LB_ETIMEOUT and leave the ctx usable.  The protocol itself is modelled on
the host in test_dataflow_model.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_common import Grid, normwise, random_field, round_to_storage  # noqa: E402
from workloads import gaussian_blob, guillotine, regular_blocks  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def make(g, q, vps, kc=None, **opt):
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    o = lb.lb_default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    return Simulation([g], [q], vps, kc_arrays=[kc], options=o)


def to_queue(sim):
    sim.step(1)
    sim.measure()
    sim.rebalance("queue")


CASES = {
    # nz, velocity, dynamics, k_c source, layout
    "nz96_disk_guillotine": (96, (0.5, 0.5, 0.0), 0, "disk", "guillotine"),
    "nz64_upwind_reversed": (64, (-0.4, 0.35, -0.2), 0, "array", "blocks"),
    "nz32_x_only": (32, (-0.5, 0.0, 0.0), 0, "disk", "guillotine"),
    "nz96_jacobi": (96, (0.5, 0.5, 0.0), 1, "array", "blocks"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_dataflow_equals_barrier_kernel_and_oracle(name):
    from paper_1310_4218_gb300 import lb
    nz, (cx, cy, cz), dyn, kcsrc, layout = CASES[name]
    nx, ny = 96, 72
    g = Grid(nx, ny, nz, cx, cy, cz, kc_disk=(kcsrc == "disk"), disk=(30, 20, 1, 2, 14),
             k_in=9, k_out=1, dynamics=dyn)
    q = round_to_storage(gaussian_blob(nx, ny, nz, (48, 36, nz / 2), 10.0, 1e-3, 71), "f32")
    kc = None
    if kcsrc == "array":
        kc = np.random.default_rng(72).integers(0, 12, size=(ny, nx)).astype(np.int32)
    vps = guillotine(nx, ny, 40, 4, 73, x_align=8) if layout == "guillotine" else \
        regular_blocks(nx, ny, 16, 12)
    a = make(g, q, vps, kc, dataflow=1)
    b = make(g, q, vps, kc)
    for s in (a, b):
        to_queue(s)
    assert a.info().dataflow == 1 and b.info().dataflow == 0
    for n in (7, 1, 12):                        # launches of several lengths
        a.step(n)
        b.step(n)
    fa, fb = a.field(0), b.field(0)
    ma, mb = a.mass_history(0), b.mass_history(0)
    a.close()
    b.close()
    assert np.array_equal(fa, fb)
    assert len(ma) == len(mb) == 21
    assert np.abs(ma - mb).max() <= 1e-12 * np.abs(mb).max()
    ref, _ = oracle.run(g.oracle(kc), q, 21)
    assert normwise(fa, ref) <= 1e-5


def test_dataflow_only_in_queue_mode():
    """With processor tables the barrier kernel runs; back in queue mode the
    dataflow kernel; the fields stay equal to a plain run throughout."""
    g = Grid(64, 48, 96, disk=(10, 10, 1, 1, 9), k_in=7, k_out=1)
    q = round_to_storage(random_field(g, 74), "f32")
    vps = regular_blocks(64, 48, 16, 8)
    a = make(g, q, vps, dataflow=1)
    b = make(g, q, vps)
    assert a.info().dataflow == 0               # static tables at create
    for strategy, n in (("queue", 5), ("greedy_blocked", 3), ("queue", 4)):
        for s in (a, b):
            s.step(1)
            s.measure()
            s.rebalance(strategy)
        assert a.info().dataflow == (1 if strategy == "queue" else 0)
        a.step(n)
        b.step(n)
    fa, fb = a.field(0), b.field(0)
    a.close()
    b.close()
    assert np.array_equal(fa, fb)


def test_dataflow_graph_replays_equal_direct_steps():
    from paper_1310_4218_gb300 import lb
    g = Grid(80, 48, 64, disk=(10, 40, 1, 2, 9), k_in=11, k_out=1)
    q = round_to_storage(gaussian_blob(80, 48, 64, (40, 24, 32), 9.0, 1e-3, 75), "f32")
    vps = regular_blocks(80, 48, 16, 8)
    a = make(g, q, vps, dataflow=1)
    to_queue(a)
    a.step(9)
    ref = a.field(0)
    a.close()
    b = make(g, q, vps, dataflow=1)
    to_queue(b)
    graph = lb.lb_graph_create(b.ctx, 3)
    for _ in range(3):
        lb.lb_graph_launch(b.ctx, graph)
    out = b.field(0)
    assert b.info().step == 10
    lb.lb_graph_destroy(b.ctx, graph)
    b.close()
    assert np.array_equal(out, ref)


def test_dataflow_wait_limit_is_reported_and_ctx_recovers():
    """A 1 ns wait limit: the first wait that does not succeed at once gives
    up, records LB_ETIMEOUT and the launch ends (no wait outlives the
    status); the next synchronising call reports it, and the one after
    finds the status clear."""
    from paper_1310_4218_gb300 import lb
    g = Grid(64, 64, 64, disk=(16, 16, 0, 0, 6), k_in=200, k_out=0)
    q = round_to_storage(random_field(g, 76), "f32")
    sim = make(g, q, regular_blocks(64, 64, 16, 16), dataflow=1, barrier_timeout_ns=1)
    sim.rebalance("queue")                      # no barrier step before: its wait would give up
    assert sim.info().dataflow == 1
    sim.step(6)
    with pytest.raises(lb.LBError) as e:
        sim.sync()
    assert e.value.status == lb.LB_ETIMEOUT
    sim.sync()
    sim.close()


def test_dataflow_two_grids_and_owned_subsets():
    """Two grids in one ctx (dependencies never cross grids), then the same
    ctx restricted to half of its VPs (lb_set_owned: the other VPs have no
    work items, so their columns have no owner in the dependency lists):
    fields equal the barrier kernel's bit for bit on every owned column."""
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    g1 = Grid(64, 48, 96, disk=(10, 10, 1, 1, 9), k_in=7, k_out=1)
    g2 = Grid(40, 56, 96, -0.5, 0.5, 0.0, disk=(20, 30, 1, 0, 8), k_in=5, k_out=1)
    q1 = round_to_storage(random_field(g1, 77), "f32")
    q2 = round_to_storage(random_field(g2, 78), "f32")
    vps = regular_blocks(64, 48, 16, 8, grid=0) + regular_blocks(40, 56, 8, 14, grid=1)

    def sim(df):
        o = lb.lb_default_options()
        o.dataflow = df
        s = Simulation([g1, g2], [q1, q2], vps, options=o)
        s.rebalance("queue")
        return s

    a, b = sim(1), sim(0)
    assert a.info().dataflow == 1
    a.step(6)
    b.step(6)
    for gi in (0, 1):
        assert np.array_equal(a.field(gi), b.field(gi))
    owned = (np.arange(len(vps)) % 2).astype(np.uint8)
    for s in (a, b):
        lb.lb_set_owned(s.ctx, owned)
    assert a.info().dataflow == 1
    a.step(5)
    b.step(5)
    for gi, g in enumerate((g1, g2)):
        fa, fb = a.field(gi), b.field(gi)
        for v, (vg, x0, y0, w, h) in enumerate(vps):
            if vg == gi and owned[v]:
                assert np.array_equal(fa[:, y0:y0 + h, x0:x0 + w], fb[:, y0:y0 + h, x0:x0 + w])
    a.close()
    b.close()
