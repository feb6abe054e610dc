"""Failure detection without a GPU fault.

Bad host inputs are refused with LB_EINVAL before anything changes, and the
ctx runs on exactly as before.  A processor count that cannot be co-resident
is refused at create (LB_ENORESIDENT).  A non-finite global sum is recorded
by the kernel in the ctx's status word, reported once by the next
synchronising call (LB_ENUMERIC), then cleared.  Nothing here traps, faults
or waits without a limit: NaN only flows through arithmetic, and the refusals
happen on the host.  (The barrier time limit has its own test in
test_gpu_parity.py.)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_common import Grid, normwise, random_field, round_to_storage, tolerance  # noqa: E402
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


def test_bad_costs_and_assignments_are_refused_and_change_nothing():
    """NaN or negative costs, and processor indices outside [0, nprocs), are
    refused; the cost averages and the table stay as they were, and the
    following steps still match the oracle."""
    from paper_1310_4218_gb300 import lb
    g = Grid(48, 40, 32, disk=(10, 10, 1, 1, 8), k_in=9)
    q = round_to_storage(random_field(g, 31), "f32")
    vps = regular_blocks(48, 40, 16, 8)
    n = len(vps)
    sim = make_sim([g], [q], vps)
    sim.step(2)
    sim.measure()
    a0, nprocs = sim.assignment()
    c0 = lb.lb_get_costs(sim.ctx, n)[0]
    for bad in ([float("nan")] + [1.0] * (n - 1), [-1.0] + [1.0] * (n - 1)):
        with pytest.raises(lb.LBError) as e:
            sim.set_costs(bad)
        assert e.value.status == lb.LB_EINVAL
    for bad in ([nprocs] + [0] * (n - 1), [-1] + [0] * (n - 1)):
        with pytest.raises(lb.LBError) as e:
            lb.lb_set_assignment(sim.ctx, bad)
        assert e.value.status == lb.LB_EINVAL
    a1, _ = sim.assignment()
    assert np.array_equal(a0, a1)
    assert np.array_equal(lb.lb_get_costs(sim.ctx, n)[0], c0)
    sim.step(3)
    out = sim.field(0)
    sim.close()
    ref, _ = oracle.run(g.oracle(), q, 5)
    assert normwise(out, ref) <= tolerance(g, 5)


def test_processors_that_cannot_be_co_resident_are_refused():
    """64 processors per SM is beyond any step kernel's co-residency limit:
    lb_create refuses before any launch."""
    from paper_1310_4218_gb300 import lb
    g = Grid(32, 32, 32, disk=(8, 8, 0, 0, 4), k_in=3)
    q = round_to_storage(random_field(g, 32), "f32")
    with pytest.raises(lb.LBError) as e:
        make_sim([g], [q], regular_blocks(32, 32, 16, 16), ctas_per_sm=64)
    assert e.value.status == lb.LB_ENORESIDENT


def test_non_finite_global_sum_is_reported_once():
    """A NaN in the field makes the step's global sum non-finite: the kernel
    records LB_ENUMERIC, the next synchronising call reports it, and the one
    after that finds the status word clear."""
    from paper_1310_4218_gb300 import lb
    g = Grid(32, 32, 32, disk=(8, 8, 0, 0, 4), k_in=3)
    q = round_to_storage(random_field(g, 33), "f32")
    q[5, 7, 9] = np.nan
    sim = make_sim([g], [q], regular_blocks(32, 32, 16, 16))
    sim.step(1)
    with pytest.raises(lb.LBError) as e:
        sim.sync()
    assert e.value.status == lb.LB_ENUMERIC
    sim.sync()
    sim.close()


@pytest.mark.parametrize("threads_hint", [0, 1, 2, 4])
def test_k_c_entries_above_the_bound_are_clamped_and_reported_once(threads_hint):
    """A k_c array with entries above LB_KC_MAX (and below 0) runs them
    clamped to 0..LB_KC_MAX: the field equals the oracle's with the clamped
    array, the next synchronising call reports LB_EKCRANGE, and the one
    after that finds the flag clear.  A small grid keeps the launch short
    (a few columns run LB_KC_MAX solves)."""
    from paper_1310_4218_gb300 import lb
    g = Grid(48, 32, 32, kc_disk=False)
    q = round_to_storage(random_field(g, 34), "f32")
    rng = np.random.default_rng(35)
    kc = rng.integers(0, 6, size=(g.ny, g.nx)).astype(np.int32)
    kc[3, 5] = lb.LB_KC_MAX + 1
    kc[20, 40] = 2 ** 31 - 1
    kc[7, 7] = -5
    kc[9, 30] = lb.LB_KC_MAX               # at the bound: no report of its own
    clamped = np.clip(kc, 0, lb.LB_KC_MAX)
    from paper_1310_4218_gb300.sim import Simulation
    o = lb.lb_default_options()
    o.threads_hint = threads_hint
    sim = Simulation([g], [q], regular_blocks(48, 32, 16, 8), kc_arrays=[kc], options=o)
    sim.step(2)
    with pytest.raises(lb.LBError) as e:
        sim.sync()
    assert e.value.status == lb.LB_EKCRANGE
    sim.sync()
    out = sim.field(0)
    # an array within the bound reports nothing
    sim.set_kc(0, clamped)
    sim.step(1)
    sim.sync()
    out3 = sim.field(0)
    sim.close()
    ref, _ = oracle.run(g.oracle(clamped), q, 2)
    assert normwise(out, ref) <= tolerance(g, 2)
    ref3, _ = oracle.run(g.oracle(clamped), q, 3)
    assert normwise(out3, ref3) <= tolerance(g, 3)
