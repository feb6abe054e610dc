"""Seeded random configurations against the FP64 oracle, whole field.

Each case draws a grid (nx, ny in 8..72; nz among 1, 2, 7, 17, 32, 33, 64,
95, 96, 100, 128), a storage/compute pair, velocities of either sign (some
with vertical advection, some on the two-neighbour stencil), r, a disk or
an array k_c, the advection or the Jacobi dynamics, a guillotine or block
VP layout, a kernel hint, stealing, the dataflow option and a strategy;
runs a few steps, measures, rebalances and runs a few more; and compares
every cell with the oracle within the precision's bound.  The draws stay
inside what the ABI accepts, so every case must run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_common import Grid, normwise, random_field, round_to_storage, tolerance  # noqa: E402
from workloads import guillotine, regular_blocks  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


NZS = [1, 2, 7, 17, 32, 33, 64, 95, 96, 100, 128]
PRECS = [("f32", "f32"), ("f32", "f32"), ("f64", "f64"), ("f64", "f32"), ("bf16", "f32")]
STRATEGIES = ["queue", "greedy", "greedy_blocked", "greedy_spatial", "refine_swap", "static",
              "auto_spatial"]


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    storage, compute = PRECS[rng.integers(len(PRECS))]
    nzs = [z for z in NZS if compute != "f64" or z <= 64]
    nz = int(rng.choice(nzs))
    nx, ny = int(rng.integers(8, 73)), int(rng.integers(8, 73))
    dynamics = int(rng.random() < 0.25)
    if rng.random() < 0.4:                       # the two-neighbour stencil
        cx = float(rng.choice([-1, 1]) * rng.choice([0.25, 0.5, 0.75]))
        cy = float(np.sign(rng.random() - 0.5) * (1.0 - abs(cx)))
        cz = 0.0
    else:
        c = rng.uniform(-1, 1, 3)
        c *= rng.uniform(0.2, 1.0) / np.abs(c).sum()
        cx, cy, cz = (float(v) for v in c)
    r = float(rng.choice([0.0, 0.1, 0.1, 0.5]))
    kc_disk = bool(rng.random() < 0.5)
    disk = (int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(-2, 3)),
            int(rng.integers(-2, 3)), int(rng.integers(2, 12)))
    g = Grid(nx, ny, nz, cx, cy, cz, r, storage, compute, kc_disk, disk,
             int(rng.integers(0, 9)), int(rng.integers(0, 3)), dynamics,
             float(rng.uniform(0.05, 1.0 / 6.0)))
    kc = None if kc_disk else rng.integers(0, 9, size=(ny, nx)).astype(np.int32)
    if rng.random() < 0.5:
        nleaves = int(rng.integers(1, 24))
        vps = guillotine(nx, ny, nleaves, 2, int(rng.integers(1 << 30)))
    else:
        vps = regular_blocks(nx, ny, int(rng.integers(1, 24)), int(rng.integers(1, 24)))
    hints = [0, 1, 2, 4] + ([3] if storage == compute == "f32" and nz in (32, 64, 96) else [])
    opt = {"threads_hint": int(rng.choice(hints)), "steal": int(rng.random() < 0.5),
           "dataflow": int(rng.random() < 0.5)}
    strategy = str(rng.choice(STRATEGIES))
    n1, n2 = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    return g, kc, vps, opt, strategy, n1, n2


@pytest.mark.parametrize("seed", range(120))
def test_random_configuration_matches_the_oracle(seed):
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    g, kc, vps, opt, strategy, n1, n2 = draw(seed)
    q = round_to_storage(random_field(g, 2000 + seed), g.storage)
    o = lb.lb_default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    sim = Simulation([g], [q], vps, kc_arrays=[kc], options=o)
    sim.step(n1)
    sim.measure()
    sim.rebalance(strategy)
    sim.step(n2)
    out = sim.field(0)
    sim.close()
    ref, _ = oracle.run(g.oracle(kc), q, n1 + n2)
    err = normwise(out, ref)
    assert err <= tolerance(g, n1 + n2), (err, g.__dict__, opt, strategy)
