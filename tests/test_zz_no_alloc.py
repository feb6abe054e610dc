"""lb_step_noalloc: the allocation-free entry point for callers whose device
memory belongs to another allocator (a framework's caching allocator, a
fixed-budget pool) and who therefore cannot let the library call cudaMalloc.
Its field must equal the ctx path's (lb_create + lb_step, same kernel) bit
for bit and agree with the FP64 oracle, call after call, for every storage
and compute type, exact and runtime column lengths, k_c arrays and the
Jacobi dynamics; its global sum must match the ctx path's; and it must
refuse inputs beyond its fixed maxima and layouts that do not tile the grid.

This file is collected last so that a run stopping at its first failure has
run every other test already."""
import numpy as np
import pytest

from gpu_common import Grid, normwise, round_to_storage, tolerance
from workloads import gaussian_blob, regular_blocks


@pytest.fixture(scope="module")
def lbmod():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_4218_gb300 import lb
    return lb


def desc(lb, g, q0_ptr, q1_ptr, kc_ptr=None):
    x0, y0, vx, vy, R = g.disk
    return lb.lb_grid_desc(g.nx, g.ny, g.nz, g.cx, g.cy, g.cz, g.r, lb.DTYPES[g.storage],
                           lb.DTYPES[g.compute], q0_ptr, q1_ptr, kc_ptr, 1 if g.kc_disk else 0,
                           x0, y0, vx, vy, R, g.k_in, g.k_out, g.dynamics, 0, g.nu)


def test_limits_are_enforced_before_any_device_work(lbmod):
    lb = lbmod
    g = Grid(257, 8192, 1)
    d = desc(lb, g, 0x1000, 0x2000)
    # 8192 VPs of 257 columns: 9 work items each, above LB_NOALLOC_MAX_ITEMS
    vps = [(0, 0, j, 257, 1) for j in range(8192)]
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_noalloc(d, vps, 0, 1)
    assert e.value.status == lb.LB_EINVAL and "work items" in str(e.value)
    g2 = Grid(100, 100, 4)
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_noalloc(desc(lb, g2, 0x1000, 0x2000), regular_blocks(100, 100, 1, 1), 0, 1)
    assert e.value.status == lb.LB_EINVAL and "nvps" in str(e.value)


def test_overlap_with_an_equal_gap_is_refused_on_a_large_grid(lbmod):
    """4096 x 2048 columns (above the old 4M-column bitmap): one strip of VPs
    shifted down a row overlaps its neighbour and leaves the top row
    uncovered; the areas still add up to the grid's, so only the overlap
    check can refuse it."""
    lb = lbmod
    g = Grid(4096, 2048, 1)
    vps = [(0, 0, 32 * s, 4096, 32) for s in range(64)]
    vps[63] = (0, 0, 32 * 63 - 1, 4096, 32)
    assert sum(v[3] * v[4] for v in vps) == 4096 * 2048
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_noalloc(desc(lb, g, 0x1000, 0x2000), vps, 0, 1)
    assert e.value.status == lb.LB_EINVAL and "overlap" in str(e.value)


def test_descriptor_checks_match_lb_create(lbmod):
    """The per-grid checks are lb_create's: kc_disk outside {0, 1}, a disk
    k_c above LB_KC_MAX and more columns than the tiling bitmap holds are
    refused."""
    lb = lbmod
    g = Grid(64, 64, 8)
    vps = regular_blocks(64, 64, 16, 16)
    d = desc(lb, g, 0x1000, 0x2000)
    d.kc_disk = 2
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_noalloc(d, vps, 0, 1)
    assert e.value.status == lb.LB_EINVAL and "kc_disk" in str(e.value)
    d = desc(lb, g, 0x1000, 0x2000)
    d.k_in = lb.LB_KC_MAX + 1
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_noalloc(d, vps, 0, 1)
    assert e.value.status == lb.LB_EINVAL and "LB_KC_MAX" in str(e.value)
    big = Grid(16384, 8193, 1)
    with pytest.raises(lb.LBError) as e:
        lb.lb_step_noalloc(desc(lb, big, 0x1000, 0x2000), [(0, 0, 0, 16384, 8193)], 0, 1)
    assert e.value.status == lb.LB_EINVAL and "LB_NOALLOC_MAX_COLUMNS" in str(e.value)


# grid, initial-field seed, VP block size; storage/compute, exact and runtime
# column lengths, a k_c array, the Jacobi dynamics
CASES = {
    "f32_nz64_disk": (Grid(96, 80, 64, disk=(20, 30, 1, 1, 14), k_in=12, k_out=1), 31, (16, 16)),
    "f32_nz40_array": (Grid(72, 56, 40, kc_disk=False), 32, (24, 8)),
    "f32_nz96_wide_disk": (Grid(64, 48, 96, disk=(10, 20, 1, 1, 9), k_in=9), 33, (32, 16)),
    "f64_nz30_disk": (Grid(48, 40, 30, storage="f64", compute="f64", disk=(8, 8, 1, 1, 9),
                           k_in=7), 34, (16, 8)),
    "f64s_f32c_nz64": (Grid(48, 40, 64, storage="f64", compute="f32", disk=(30, 8, 1, 1, 9),
                            k_in=5), 35, (16, 8)),
    "bf16_nz64_disk": (Grid(64, 48, 64, storage="bf16", disk=(20, 20, 1, 1, 10), k_in=6), 36,
                       (16, 16)),
    "f32_nz96_jacobi": (Grid(64, 48, 96, dynamics=1, disk=(30, 20, 1, 1, 10), k_in=5), 37,
                        (32, 16)),
}


def _kc_array(g, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 9, size=(g.ny, g.nx)).astype(np.int32)


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_equals_ctx_path_and_oracle_on_consecutive_calls(lbmod, name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    lb = lbmod
    from paper_1310_4218_gb300.sim import Simulation

    g, seed, (bw, bh) = CASES[name]
    q = round_to_storage(gaussian_blob(g.nx, g.ny, g.nz, (g.nx / 2, g.ny / 2, g.nz / 2),
                                       g.nx / 6, 1e-3, seed), g.storage)
    vps = regular_blocks(g.nx, g.ny, bw, bh)
    kc = None if g.kc_disk else _kc_array(g, seed)

    # the existing entry points: lb_create + lb_step, static placement
    sim = Simulation([g], [q], vps, kc_arrays=[kc])
    sim.step(3)
    ref1 = sim.field(0)
    m1 = sim.mass(0)[0]
    sim.step(2)
    ref2 = sim.field(0)
    m2 = sim.mass(0)[0]
    sim.close()

    dev = torch.device("cuda:0")
    dt = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16}[g.storage]
    b0 = torch.as_tensor(q).to(device=dev, dtype=dt).contiguous()
    b1 = torch.empty_like(b0)
    kc_t = None if kc is None else torch.as_tensor(kc).to(dev)
    kp = None if kc_t is None else kc_t.data_ptr()
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize(dev)
    # first call: 3 steps from b0, result in b1 (odd count)
    s1 = lb.lb_step_noalloc(desc(lb, g, b0.data_ptr(), b1.data_ptr(), kp), vps, 0, 3, stream)
    out1 = b1.double().cpu().numpy()
    # second call: 2 more steps from b1, result back in b1 (even count)
    s2 = lb.lb_step_noalloc(desc(lb, g, b1.data_ptr(), b0.data_ptr(), kp), vps, 3, 2, stream)
    out2 = b1.double().cpu().numpy()

    # the same kernel on the same columns: the fields agree bit for bit
    assert np.array_equal(out1, ref1) and np.array_equal(out2, ref2)
    # the global sum adds the same stored values (in another order)
    assert abs(s1 - m1) <= 1e-12 * abs(m1)
    assert abs(s2 - m2) <= 1e-12 * abs(m2)
    # and both agree with the FP64 oracle
    o1, _ = oracle.run(g.oracle(kc), q, 3)
    o2, _ = oracle.run(g.oracle(kc), o1, 2, t0=3)
    assert normwise(out1, o1) <= tolerance(g, 3)
    assert normwise(out2, o2) <= tolerance(g, 5)
