"""Sharded run on the host: two ranks (gloo, spawned processes) split the
grid into blocks, exchange halo columns before every step, reduce the
compensated global sum, rebalance VPs across ranks from their summed
measured costs, and migrate the moved VPs' columns.  The local compute of
a rank is the FP64 oracle over the whole grid, of which the rank keeps its
owned columns -- so the assembled field must equal the single-process
oracle run bit for bit, and the global sum must match the oracle's.  No
GPU is involved; the GPU side of the same protocol (owned masks, packing
kernels) is tested in test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import OracleGrid  # noqa: E402
from paper_1310_4218_gb300 import shard  # noqa: E402
from workloads import gaussian_blob, regular_blocks  # noqa: E402


class G:
    """Grid description: 48 x 40 x 16, advection (0.5, 0.5), a k_c disk in
    the left half (rank 0's block) that moves one cell per step."""
    nx, ny, nz = 48, 40, 16
    cx, cy, cz, r = 0.5, 0.5, 0.0, 0.1
    storage = compute = "f64"
    kc_disk, disk, k_in, k_out = True, (10, 20, 1, 0, 8), 12, 1
    dynamics, nu = 0, 1.0 / 7.0


def og():
    return OracleGrid(G.nx, G.ny, G.nz, G.cx, G.cy, G.cz, G.r, True, G.disk, G.k_in, G.k_out)


def initial():
    return gaussian_blob(G.nx, G.ny, G.nz, (24.0, 20.0, 8.0), 7.0, 1e-3, 41)


class OracleStepper:
    """A rank's compute for the test: one oracle step of the whole local
    field, of which only the owned columns are kept (the others stay as
    they were, as on a GPU that does not run those VPs)."""

    def __init__(self, vps):
        self.q = initial().copy()
        self.vps = vps
        self.t = 0
        self.mask = np.ones(len(vps), dtype=np.uint8)
        self.cols = np.zeros(G.nx * G.ny, dtype=bool)

    def set_owned(self, mask):
        self.mask = np.asarray(mask, dtype=np.uint8)
        self.cols[:] = False
        for v, vp in enumerate(self.vps):
            if self.mask[v]:
                self.cols[shard.vp_cells(vp, G.nx)] = True

    def step(self, n):
        for _ in range(n):
            new, _ = oracle.run(og(), self.q, 1, t0=self.t)
            flat, nflat = self.q.reshape(G.nz, -1), new.reshape(G.nz, -1)
            flat[:, self.cols] = nflat[:, self.cols]
            self.t += 1

    def pack(self, g, cells):
        return torch.from_numpy(self.q.reshape(G.nz, -1)[:, cells].copy())

    def unpack(self, g, cells, data):
        self.q.reshape(G.nz, -1)[:, cells] = data.numpy()

    def alloc(self, g, n):
        return torch.empty((G.nz, n), dtype=torch.float64)

    def partial_mass(self, g):
        return oracle.compensated_sum(self.q.reshape(G.nz, -1)[:, self.cols]), 0.0

    def costs(self):
        kc = oracle.kc_field(og(), self.t)
        c = np.zeros(len(self.vps))
        for v, (_, x0, y0, w, h) in enumerate(self.vps):
            if self.mask[v]:
                c[v] = float(kc[y0:y0 + h, x0:x0 + w].sum()) * G.nz + w * h
        return c


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        vps = regular_blocks(G.nx, G.ny, 12, 10)
        st = OracleStepper(vps)
        run = shard.ShardedRun(st, vps, [G], shard.TorchComm())
        owner0 = run.owner.copy()
        run.step(4)
        m4 = run.mass(0)
        moved = run.rebalance("greedy")
        owner1 = run.owner.copy()
        run.step(4)
        m8 = run.mass(0)
        # assemble the owned columns of every rank on every rank
        full = torch.from_numpy(np.where(st.cols[None, :], st.q.reshape(G.nz, -1), 0.0))
        dist.all_reduce(full)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), field=full.numpy(),
                 owner0=owner0, owner1=owner1, m4=np.array(m4), m8=np.array(m8),
                 moved=moved, recv=sum(len(c) for c in run.plan.recv.values()))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_sharded_run_equals_the_oracle(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    r0, r1 = (np.load(tmp_path / ("rank%d.npz" % r)) for r in range(2))
    # both ranks hold the same owner maps: a 2 x 1 block split, then the
    # balancer's map, which moved VPs off the loaded left block
    assert np.array_equal(r0["owner0"], r1["owner0"]) and np.array_equal(r0["owner1"], r1["owner1"])
    assert set(r0["owner0"].tolist()) == {0, 1}
    assert int(r0["moved"]) == int(np.sum(r0["owner0"] != r0["owner1"])) > 0
    assert int(r0["recv"]) > 0 and int(r1["recv"]) > 0
    # the assembled field is the oracle's, bit for bit
    ref4, mass4 = oracle.run(og(), initial(), 4)
    ref8, mass8 = oracle.run(og(), ref4, 4, t0=4)
    assert np.array_equal(r0["field"], ref8.reshape(G.nz, -1))
    assert np.array_equal(r0["field"], r1["field"])
    # the folded FP64 partial sums are the global sum, on every rank
    for r in (r0, r1):
        assert abs(float(r["m4"][0]) + float(r["m4"][1]) - mass4[-1]) <= 1e-12 * abs(mass4[-1])
        assert abs(float(r["m8"][0]) + float(r["m8"][1]) - mass8[-1]) <= 1e-12 * abs(mass8[-1])


def test_halo_plan_is_symmetric_and_covers_every_read():
    """Host plans for four ranks: what rank r receives from p is what p
    sends to r, and every column a rank's VPs read outside themselves is
    either its own or received."""
    vps = regular_blocks(G.nx, G.ny, 12, 10)
    owner = shard.block_owners(vps, [G], 4)
    assert sorted(set(owner.tolist())) == [0, 1, 2, 3]
    plans = [shard.HaloPlan(vps, [G], owner, r, 4) for r in range(4)]
    co = shard.cell_owners(vps, [G], owner)[0]
    for r in range(4):
        for (g, p), cells in plans[r].recv.items():
            assert np.array_equal(cells, plans[p].send[(g, r)])
            assert (co[cells] == p).all()
        have = set(np.flatnonzero(co == r).tolist())
        for (g, p), cells in plans[r].recv.items():
            have |= set(cells.tolist())
        for v, vp in enumerate(vps):
            if owner[v] == r:
                assert set(shard.halo_cells(vp, G).tolist()) <= have


def test_fold_partials_is_order_fixed_and_compensated():
    parts = [(1e16, 0.0), (1.0, 0.0), (-1e16, 0.0), (1.0, 1e-17)]
    s, c = shard.fold_partials(parts)
    assert s + c == 2.0
    assert shard.rank_grid(6) == (3, 2) and shard.rank_grid(7) == (7, 1)
