"""Load measurement under different co-residency (Sec. V, Table I): the
default concurrent steps with 1, 2 or 4 processors (CTAs) sharing each SM,
and serialized measurement steps (lb_step_serial: one working warp per
processor).  Each mode must produce the oracle's field and a measured cost
for every VP; serialized steps give the same field as concurrent ones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_common import Grid, normwise, round_to_storage  # noqa: E402
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


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("ctas", [1, 2, 4])
def test_processors_sharing_an_sm(ctas, wide):
    """nz 96 grids on the half-warp (narrow VPs) and twin (wide VPs) kernels
    with 1, 2 or 4 processors per SM: 1/ctas of the threads per processor,
    ctas times the processors; fields equal the oracle's and every VP gets
    a measured cost."""
    nx = 64 if wide else 56
    g = Grid(nx, 40, 96, disk=(20, 20, 1, 1, 9), k_in=11, k_out=1)
    q = round_to_storage(gaussian_blob(nx, 40, 96, (nx / 2, 20, 48), 9.0, 1e-3, 61), "f32")
    vps = regular_blocks(nx, 40, 16 if wide else 8, 8)
    sim = make(g, q, vps, ctas_per_sm=ctas)
    info = sim.info()
    assert info.nprocs == ctas * info.nsm
    sim.step(3)
    cost, _ = sim.measure()
    assert (cost > 0).all()
    sim.rebalance("greedy_blocked")
    sim.step(2)
    out = sim.field(0)
    sim.close()
    ref, _ = oracle.run(g.oracle(), q, 5)
    assert normwise(out, ref) <= 1e-5


@pytest.mark.parametrize("threads_hint", [0, 2, 4])
def test_serial_measurement_steps(threads_hint):
    """Serialized steps (one working warp per processor) leave the same field
    as concurrent steps, bit for bit, and measure every VP."""
    g = Grid(48, 40, 32, kc_disk=False)
    rng = np.random.default_rng(62)
    kc = rng.integers(1, 9, size=(40, 48)).astype(np.int32)
    q = round_to_storage(gaussian_blob(48, 40, 32, (24, 20, 16), 8.0, 1e-3, 62), "f32")
    vps = guillotine(48, 40, 20, 4, 63)
    from paper_1310_4218_gb300 import lb
    a = make(g, q, vps, kc, threads_hint=threads_hint)
    b = make(g, q, vps, kc, threads_hint=threads_hint)
    a.step(2)
    lb.lb_step_serial(b.ctx, 1)
    cost, _ = b.measure()
    assert (cost > 0).all()
    b.step(1)
    fa, fb = a.field(0), b.field(0)
    a.close()
    b.close()
    assert np.array_equal(fa, fb)
    ref, _ = oracle.run(g.oracle(kc), q, 2)
    assert normwise(fa, ref) <= 1e-5


def test_serial_steps_refused_on_paired_warps():
    from paper_1310_4218_gb300 import lb
    g = Grid(32, 32, 32, disk=(8, 8, 0, 0, 4), k_in=3)
    q = round_to_storage(gaussian_blob(32, 32, 32, (16, 16, 16), 5.0, 1e-3, 64), "f32")
    sim = make(g, q, regular_blocks(32, 32, 16, 16), threads_hint=3)
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_serial(sim.ctx, 1)
    assert e.value.status == lb.LB_ESTATE
    sim.close()
