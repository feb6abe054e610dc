"""lb_step_noalloc: the allocation-free entry point for callers whose device
memory belongs to another allocator (a framework's caching allocator, a
fixed-budget pool) and who therefore cannot let the library call cudaMalloc.
It must produce the same fields and global sum as the ctx path (lb_create +
lb_step), call after call, and refuse inputs beyond its fixed maxima.

This file is collected last so that a run stopping at its first failure has
run every other test already."""
import numpy as np
import pytest

from gpu_common import Grid, normwise, round_to_storage
from workloads import gaussian_blob, regular_blocks


@pytest.fixture(scope="module")
def lbmod():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1310_4218_gb300 import lb
    return lb


def desc(lb, g, q0_ptr, q1_ptr):
    x0, y0, vx, vy, R = g.disk
    return lb.lb_grid_desc(g.nx, g.ny, g.nz, g.cx, g.cy, g.cz, g.r, lb.DTYPES[g.storage],
                           lb.DTYPES[g.compute], q0_ptr, q1_ptr, None, 1, x0, y0, vx, vy, R,
                           g.k_in, g.k_out)


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


@pytest.mark.gpu
def test_noalloc_matches_ctx_path_on_consecutive_calls(lbmod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lb = lbmod
    from paper_1310_4218_gb300.sim import Simulation

    g = Grid(96, 80, 64, disk=(20, 30, 1, 1, 14), k_in=12, k_out=1)
    q = round_to_storage(gaussian_blob(96, 80, 64, (48, 40, 32), 12.0, 1e-3, 31), "f32")
    vps = regular_blocks(96, 80, 16, 16)

    # the existing entry points: lb_create + lb_step, static placement
    sim = Simulation([g], [q], vps)
    sim.step(3)
    ref1 = sim.field(0)
    m1 = sim.mass(0)[0]
    sim.step(2)
    ref2 = sim.field(0)
    m2 = sim.mass(0)[0]
    sim.close()

    dev = torch.device("cuda:0")
    b0 = torch.as_tensor(q).to(device=dev, dtype=torch.float32).contiguous()
    b1 = torch.empty_like(b0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize(dev)
    # first call: 3 steps from b0, result in b1 (odd count)
    s1 = lb.lb_step_noalloc(desc(lb, g, b0.data_ptr(), b1.data_ptr()), vps, 0, 3, stream)
    out1 = b1.double().cpu().numpy()
    # second call: 2 more steps from b1, result back in b1 (even count)
    s2 = lb.lb_step_noalloc(desc(lb, g, b1.data_ptr(), b0.data_ptr()), vps, 3, 2, stream)
    out2 = b1.double().cpu().numpy()

    assert normwise(out1, ref1) <= 1e-5
    assert normwise(out2, ref2) <= 1e-5
    assert abs(s1 - m1) <= 1e-12 * abs(m1)
    assert abs(s2 - m2) <= 1e-12 * abs(m2)
