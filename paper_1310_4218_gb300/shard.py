"""Sharding the step across ranks: one process per GPU, each owning a set of
VPs -- the paper's processors of a distributed run (Sec. III, Fig. 2) and
the migration of VPs between them (Sec. VI).

Every rank holds the whole grid's field buffers (cheap next to an HBM of
280 GB) but runs only the VPs it owns (`lb_set_owned`).  Before each step
it receives the upwind halo columns of its VPs that other ranks own, so a
step reads only columns that are current; columns that are neither owned
nor halo may be stale and are never read.  The exchange moves packed
columns (`lb_pack_columns` / `lb_unpack_columns`) with point-to-point
sends; the global sum combines every rank's compensated FP64 partial
(sum, comp) in rank order; a rebalance sums the ranks' measured VP costs
(each rank measures only its own VPs), runs the library's host balancer
(`lb_plan`) over ranks -- identical on every rank, since its inputs are --
and moves each migrated VP's columns from its old owner to its new one.

The stepper (the local compute of one rank) and the communicator are
passed in: `GPUStepper` wraps a Simulation; `TorchComm` wraps
torch.distributed (NCCL between GPUs, gloo on the host).
"""
import numpy as np

from . import lb as L

# -------------------------------------------------------------- ownership


def rank_grid(nranks):
    """px x py ranks, px * py = nranks, as square as possible (px >= py)."""
    py = int(np.floor(np.sqrt(nranks)))
    while nranks % py:
        py -= 1
    return nranks // py, py


def block_owners(vps, grids, nranks):
    """2D block split of every grid: rank (bx, by) of a px x py arrangement
    owns the VPs whose centre lies in its block.  Returns owner[nvps]."""
    px, py = rank_grid(nranks)
    owner = np.empty(len(vps), dtype=np.int32)
    for v, (g, x0, y0, w, h) in enumerate(vps):
        gr = grids[g]
        bx = min(int((x0 + w / 2.0) * px / gr.nx), px - 1)
        by = min(int((y0 + h / 2.0) * py / gr.ny), py - 1)
        owner[v] = by * px + bx
    return owner


def cell_owners(vps, grids, owner):
    """Per grid, the rank owning each column (int32 [ny * nx])."""
    out = [np.full(g.nx * g.ny, -1, dtype=np.int32) for g in grids]
    for v, (g, x0, y0, w, h) in enumerate(vps):
        m = out[g].reshape(grids[g].ny, grids[g].nx)
        m[y0:y0 + h, x0:x0 + w] = owner[v]
    return out


def vp_cells(vp, nx):
    """Column indices j * nx + i of a VP, row by row."""
    _, x0, y0, w, h = vp
    jj, ii = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
    return (jj * nx + ii).ravel().astype(np.int32)


def halo_cells(vp, g):
    """Columns outside the VP that one step of it reads: the upwind column
    and row of the advection (the downwind ones too for a velocity of the
    other sign; both sides for the Jacobi sweep), periodic in x and y."""
    _, x0, y0, w, h = vp
    nx, ny = g.nx, g.ny
    jac = getattr(g, "dynamics", 0) == 1
    xs, ys = [], []
    if jac or g.cx > 0:
        xs.append((x0 - 1) % nx)
    if jac or g.cx < 0:
        xs.append((x0 + w) % nx)
    if jac or g.cy > 0:
        ys.append((y0 - 1) % ny)
    if jac or g.cy < 0:
        ys.append((y0 + h) % ny)
    cells = [j * nx + i for i in xs for j in range(y0, y0 + h)]
    cells += [j * nx + i for j in ys for i in range(x0, x0 + w)]
    return np.asarray(cells, dtype=np.int32)


class HaloPlan:
    """Which columns each rank sends to / receives from each other rank
    before a step, for one owner map.  recv[(grid, peer)] and
    send[(grid, peer)] are sorted column indices; a rank's send list to a
    peer equals that peer's receive list from it (both are computed from
    the same global owner map)."""

    def __init__(self, vps, grids, owner, rank, nranks):
        co = cell_owners(vps, grids, owner)
        need = {}                                   # (rank, grid, peer) -> set of cells
        for v, vp in enumerate(vps):
            g = vp[0]
            r = int(owner[v])
            h = halo_cells(vp, grids[g])
            for c in h[co[g][h] != r]:
                need.setdefault((r, g, int(co[g][c])), set()).add(int(c))
        self.recv, self.send = {}, {}
        for (r, g, p), cells in need.items():
            arr = np.asarray(sorted(cells), dtype=np.int32)
            if r == rank:
                self.recv[(g, p)] = arr
            if p == rank:
                self.send[(g, r)] = arr
        self.peers = sorted({p for (_, p) in self.recv} | {p for (_, p) in self.send})


def fold_partials(parts):
    """Neumaier sum of (sum, comp) partials in the given (rank) order: the
    same FP64 value on every rank."""
    s = c = 0.0
    for ps, pc in parts:
        for v in (ps, pc):
            t = s + v
            c += (s - t) + v if abs(s) >= abs(v) else (v - t) + s
            s = t
    return s, c


# -------------------------------------------------------------- the run


class ShardedRun:
    """One rank's share of a sharded run.

    stepper: set_owned(mask), step(n), pack(grid, cells) -> array [nz, n],
    unpack(grid, cells, data), alloc(grid, n) -> empty [nz, n] receive
    buffer, partial_mass(grid) -> (sum, comp), costs() -> float64 [nvps]
    (measured for owned VPs, 0 elsewhere).
    comm: rank, size, exchange(sends, recvs, alloc) (point-to-point, both
    dicts by peer), all_gather_f64(array) -> [size, ...],
    all_reduce_sum_f64(array)."""

    def __init__(self, stepper, vps, grids, comm, owner=None):
        self.stepper, self.vps, self.grids, self.comm = stepper, list(vps), list(grids), comm
        self.owner = (np.asarray(owner, dtype=np.int32) if owner is not None
                      else block_owners(self.vps, self.grids, comm.size))
        self.history = []
        self._apply_owner()

    def _apply_owner(self):
        self.stepper.set_owned((self.owner == self.comm.rank).astype(np.uint8))
        self.plan = HaloPlan(self.vps, self.grids, self.owner, self.comm.rank, self.comm.size)

    def exchange(self):
        """Receive the halo columns of this rank's VPs from their owners."""
        sends = {}
        for (g, p), cells in self.plan.send.items():
            sends.setdefault(p, []).append((g, cells, self.stepper.pack(g, cells)))
        recvs = {}
        for (g, p), cells in self.plan.recv.items():
            recvs.setdefault(p, []).append((g, cells))
        got = self.comm.exchange(sends, recvs, self.stepper.alloc)
        for p, items in got.items():
            for (g, cells, data) in items:
                self.stepper.unpack(g, cells, data)

    def step(self, n):
        for _ in range(n):
            self.exchange()
            self.stepper.step(1)

    def mass(self, grid=0):
        """Global compensated FP64 sum of the latest field: the ranks'
        partials over their owned columns, folded in rank order."""
        ps, pc = self.stepper.partial_mass(grid)
        parts = self.comm.all_gather_f64(np.array([ps, pc], dtype=np.float64))
        return fold_partials([tuple(x) for x in parts])

    def rebalance(self, strategy="greedy"):
        """Sum the ranks' measured costs, re-map VPs to ranks with the
        library's balancer and migrate the VPs whose owner changed.
        Returns the number of migrated VPs."""
        costs = self.comm.all_reduce_sum_f64(np.asarray(self.stepper.costs(), dtype=np.float64))
        new, migrations, pred = L.lb_plan(strategy, costs, self.comm.size, self.owner)
        new = np.asarray(new, dtype=np.int32)
        self.migrate(new)
        self.history.append({"migrations": int(migrations), "predicted_max_over_mean": pred})
        return int(migrations)

    def migrate(self, new_owner):
        """Move the columns of every VP whose owner changes from its old
        owner to its new one, then switch to the new owner map."""
        rank = self.comm.rank
        sends, recvs = {}, {}
        for v, vp in enumerate(self.vps):
            a, b = int(self.owner[v]), int(new_owner[v])
            if a == b:
                continue
            cells = vp_cells(vp, self.grids[vp[0]].nx)
            if a == rank:
                sends.setdefault(b, []).append((vp[0], cells, self.stepper.pack(vp[0], cells)))
            if b == rank:
                recvs.setdefault(a, []).append((vp[0], cells))
        got = self.comm.exchange(sends, recvs, self.stepper.alloc)
        for p, items in got.items():
            for (g, cells, data) in items:
                self.stepper.unpack(g, cells, data)
        self.owner = np.asarray(new_owner, dtype=np.int32)
        self._apply_owner()


# -------------------------------------------------------------- adapters


class TorchComm:
    """torch.distributed as the communicator: NCCL for CUDA tensors, gloo
    for host tensors.  exchange() posts every send and receive of a round
    at once (batch_isend_irecv), in a fixed order on both sides."""

    def __init__(self, device=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.rank, self.size = dist.get_rank(), dist.get_world_size()
        self.device = device

    def _t(self, a):
        t = a if isinstance(a, self.torch.Tensor) else self.torch.from_numpy(np.ascontiguousarray(a))
        return t.to(self.device) if self.device is not None else t

    def exchange(self, sends, recvs, alloc):
        ops, out = [], {}
        for p in sorted(sends):
            for (_, _, data) in sends[p]:
                ops.append(self.dist.P2POp(self.dist.isend, self._t(data).contiguous(), p))
        for p in sorted(recvs):
            out[p] = []
            for (g, cells) in recvs[p]:
                buf = alloc(g, len(cells))
                ops.append(self.dist.P2POp(self.dist.irecv, buf, p))
                out[p].append((g, cells, buf))
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()
        return out

    def all_gather_f64(self, a):
        t = self._t(np.asarray(a, dtype=np.float64))
        outs = [self.torch.empty_like(t) for _ in range(self.size)]
        self.dist.all_gather(outs, t)
        return np.stack([o.cpu().numpy() for o in outs])

    def all_reduce_sum_f64(self, a):
        t = self._t(np.asarray(a, dtype=np.float64))
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return t.cpu().numpy()


class GPUStepper:
    """One rank's compute: a Simulation over the whole grid that runs only
    the owned VPs; columns move through device buffers packed by the
    library's kernels on the ctx stream."""

    def __init__(self, sim):
        import torch
        self.sim, self.torch = sim, torch
        self._idx = {}
        self.mask = np.ones(len(sim.vps), dtype=np.uint8)

    def nz(self, grid):
        return self.sim.grids[grid].nz

    def torch_dtype(self, grid):
        from .sim import _TORCH
        return _TORCH[self.sim.grids[grid].storage]

    def _cells(self, cells):
        """Device copy of an index array, cached per array object (the cache
        holds the array, so its id is not reused while cached)."""
        hit = self._idx.get(id(cells))
        if hit is not None and hit[0] is cells:
            return hit[1]
        if len(self._idx) > 256:
            self._idx.clear()
        t = self.torch.as_tensor(np.ascontiguousarray(cells, dtype=np.int32)).to(self.sim.device)
        self._idx[id(cells)] = (cells, t)
        return t

    def set_owned(self, mask):
        self.mask = np.asarray(mask, dtype=np.uint8)
        L.lb_set_owned(self.sim.ctx, self.mask)

    def alloc(self, grid, n):
        return self.torch.empty((self.nz(grid), n), dtype=self.torch_dtype(grid),
                                device=self.sim.device)

    def step(self, n):
        self.sim.step(n)

    def pack(self, grid, cells):
        idx = self._cells(cells)
        buf = self.alloc(grid, len(cells))
        L.lb_pack_columns(self.sim.ctx, grid, idx.data_ptr(), len(cells), buf.data_ptr())
        self.sim.stream.synchronize()
        return buf

    def unpack(self, grid, cells, data):
        idx = self._cells(cells)
        data = data.contiguous()
        self.sim.stream.wait_stream(self.torch.cuda.current_stream(self.sim.device))
        L.lb_unpack_columns(self.sim.ctx, grid, idx.data_ptr(), len(cells), data.data_ptr())
        data.record_stream(self.sim.stream)
        idx.record_stream(self.sim.stream)

    def partial_mass(self, grid):
        return self.sim.mass(grid)

    def costs(self):
        cost, _ = self.sim.measure()
        return cost * self.mask
