"""The GPU side of a sharded run, on one GPU: two ctxs over the same grid,
each running the VPs one rank owns (lb_set_owned), with the halo columns
moved between them by the packing kernels (lb_pack_columns /
lb_unpack_columns) before every step and a VP migration half way.  The
owned columns of the two ctxs together must equal one ctx running every VP
bit for bit (the same kernel computes every column the same way), match the
FP64 oracle, and their partial global sums must fold to the whole sum.  The
two ctxs run one after the other on one stream: no kernel waits on another.
The multi-process protocol around these calls is tested on the host in
test_shard_gloo.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from gpu_common import Grid, normwise, round_to_storage  # noqa: E402
from workloads import gaussian_blob, regular_blocks  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def owned_columns(vps, owner, rank, nx):
    from paper_1310_4218_gb300 import shard
    cols = [shard.vp_cells(vp, nx) for v, vp in enumerate(vps) if owner[v] == rank]
    return np.concatenate(cols)


@pytest.mark.parametrize("threads_hint", [0, 2])
def test_two_ctx_shards_equal_one_ctx_and_the_oracle(threads_hint):
    from paper_1310_4218_gb300 import lb, shard
    from paper_1310_4218_gb300.sim import Simulation
    g = Grid(64, 48, 32, disk=(12, 20, 1, 1, 9), k_in=14, k_out=1)
    q = round_to_storage(gaussian_blob(64, 48, 32, (32, 24, 16), 9.0, 1e-3, 51), "f32")
    vps = regular_blocks(64, 48, 16, 12)
    opt = lb.lb_default_options()
    opt.threads_hint = threads_hint

    whole = Simulation([g], [q], vps, options=opt)
    parts = [Simulation([g], [q], vps, options=opt) for _ in range(2)]
    st = [shard.GPUStepper(s) for s in parts]
    owner = shard.block_owners(vps, [g], 2)

    def apply(owner):
        for r in range(2):
            st[r].set_owned((owner == r).astype(np.uint8))
        return [shard.HaloPlan(vps, [g], owner, r, 2) for r in range(2)]

    def exchange(plans):
        for r in range(2):
            for (gi, p), cells in plans[r].send.items():
                st[p].unpack(gi, cells, st[r].pack(gi, cells))

    plans = apply(owner)
    for _ in range(5):
        exchange(plans)
        for s in st:
            s.step(1)
        whole.step(1)
    # migrate three of rank 0's VPs to rank 1
    new = owner.copy()
    moved = np.flatnonzero(owner == 0)[:3]
    new[moved] = 1
    for v in moved:
        cells = shard.vp_cells(vps[v], g.nx)
        st[1].unpack(0, cells, st[0].pack(0, cells))
    plans = apply(new)
    for _ in range(4):
        exchange(plans)
        for s in st:
            s.step(1)
        whole.step(1)

    ref = whole.field(0).reshape(g.nz, -1)
    got = np.zeros_like(ref)
    for r in range(2):
        cols = owned_columns(vps, new, r, g.nx)
        got[:, cols] = parts[r].field(0).reshape(g.nz, -1)[:, cols]
    assert np.array_equal(got, ref)
    o, _ = oracle.run(g.oracle(), q, 9)
    assert normwise(got.reshape(o.shape), o) <= 1e-5
    total = shard.fold_partials([parts[0].mass(0), parts[1].mass(0)])
    m = whole.mass(0)
    assert abs((total[0] + total[1]) - (m[0] + m[1])) <= 1e-12 * abs(m[0])
    for s in parts + [whole]:
        s.close()


def test_out_of_range_column_is_skipped_and_reported():
    """A column index outside the grid is skipped on the device (no access)
    and reported once as LB_EINVAL by the next synchronising call; the
    valid columns of the same call are copied."""
    from paper_1310_4218_gb300 import lb
    from paper_1310_4218_gb300.sim import Simulation
    g = Grid(32, 32, 16, disk=(8, 8, 0, 0, 4), k_in=3)
    q = round_to_storage(gaussian_blob(32, 32, 16, (16, 16, 8), 5.0, 1e-3, 52), "f32")
    sim = Simulation([g], [q], regular_blocks(32, 32, 16, 16))
    dev = torch.device("cuda:0")
    cells = torch.tensor([5, 32 * 32, -1, 7], dtype=torch.int32, device=dev)
    buf = torch.full((16, 4), -7.0, dtype=torch.float32, device=dev)
    lb.lb_pack_columns(sim.ctx, 0, cells.data_ptr(), 4, buf.data_ptr())
    with pytest.raises(lb.LBError) as e:
        sim.sync()
    assert e.value.status == lb.LB_EINVAL
    sim.sync()
    b = buf.cpu().numpy()
    f = q.reshape(16, -1)
    assert np.array_equal(b[:, 0], f[:, 5].astype(np.float32))
    assert np.array_equal(b[:, 3], f[:, 7].astype(np.float32))
    assert (b[:, 1] == -7.0).all() and (b[:, 2] == -7.0).all()
    sim.close()
