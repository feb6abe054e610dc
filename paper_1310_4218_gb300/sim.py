"""A ctx with its device buffers: allocation through PyTorch, all steps in
liblb.so.

`Simulation` takes grid descriptions (any objects with the attributes nx,
ny, nz, cx, cy, cz, r, storage, compute, kc_disk, disk, k_in, k_out), their
initial fields and a VP layout; it allocates the ping-pong buffers and the
k_c arrays as torch tensors on one CUDA device and drives the C ABI.
"""
import numpy as np
import torch

from . import lb as L

_TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


class Simulation:
    def __init__(self, grids, fields, vps, kc_arrays=None, options=None, device="cuda:0",
                 stream=None):
        self.device = torch.device(device)
        self.options = options
        self.grids = list(grids)
        self.vps = list(vps)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.bufs, self.kc = [], []
        descs = []
        with torch.cuda.device(self.device):
            for gi, g in enumerate(self.grids):
                dt = _TORCH[g.storage]
                pitch = getattr(g, "pitch", 0) or g.nx
                src = torch.as_tensor(np.asarray(fields[gi], dtype=np.float64)).to(
                    device=self.device, dtype=dt)
                # rows of `pitch` elements; the padding columns stay zero
                q0 = torch.zeros((g.nz, g.ny, pitch), dtype=dt, device=self.device)
                q0[:, :, :g.nx] = src.reshape(g.nz, g.ny, g.nx)
                q1 = torch.zeros_like(q0)
                self.bufs.append((q0, q1))
                kc_t = None
                if not g.kc_disk:
                    kc_t = torch.as_tensor(np.ascontiguousarray(kc_arrays[gi], dtype=np.int32)).to(
                        self.device)
                self.kc.append(kc_t)
                x0, y0, vx, vy, R = g.disk
                descs.append(L.lb_grid_desc(
                    g.nx, g.ny, g.nz, g.cx, g.cy, g.cz, g.r, L.DTYPES[g.storage],
                    L.DTYPES[g.compute], q0.data_ptr(), q1.data_ptr(),
                    kc_t.data_ptr() if kc_t is not None else None, 1 if g.kc_disk else 0,
                    x0, y0, vx, vy, R, g.k_in, g.k_out, getattr(g, "dynamics", 0), 0,
                    getattr(g, "nu", 1.0 / 7.0)))
                descs[-1].pitch = 0 if pitch == g.nx else pitch
            torch.cuda.synchronize(self.device)
            self.ctx = L.lb_create(descs, self.vps, options, self.stream.cuda_stream)
        self.nvps = len(self.vps)

    # -- stepping and balancing (Fig. 2: steps, measurement, MPI_Migrate)
    def step(self, n):
        L.lb_step(self.ctx, n)

    def measure(self):
        return L.lb_measure_loads(self.ctx, self.nvps)

    def rebalance(self, strategy):
        return L.lb_rebalance(self.ctx, strategy)

    def set_costs(self, costs):
        L.lb_set_costs(self.ctx, costs)

    def assignment(self):
        return L.lb_get_assignment(self.ctx, self.nvps)

    def set_kc(self, grid, kc_array):
        t = torch.as_tensor(np.ascontiguousarray(kc_array, dtype=np.int32)).to(self.device)
        # the copy ran on torch's current stream; the ctx stream reads the array
        torch.cuda.current_stream(self.device).synchronize()
        L.lb_set_kc(self.ctx, grid, t.data_ptr())
        # both arrays are read on the ctx stream: steps enqueued before this
        # call may still read the old one, so neither block may be reused
        # until the work queued there when it is freed has finished
        t.record_stream(self.stream)
        if self.kc[grid] is not None:
            self.kc[grid].record_stream(self.stream)
        self.kc[grid] = t

    def info(self):
        return L.lb_get_info(self.ctx)

    def sync(self):
        L.lb_sync(self.ctx)

    # -- results
    def field_tensor(self, grid=0):
        """The buffer holding the latest field of `grid`, (nz, ny, nx): a
        strided view when the rows are padded."""
        ptr = L.lb_current_field(self.ctx, grid)
        q0, q1 = self.bufs[grid]
        g = self.grids[grid]
        return (q0 if q0.data_ptr() == ptr else q1)[:, :, :g.nx]

    def field(self, grid=0):
        """Latest field of `grid` as float64 numpy (nz, ny, nx)."""
        L.lb_sync(self.ctx)
        return self.field_tensor(grid).to(torch.float64).cpu().numpy()

    def mass(self, grid=0):
        return L.lb_mass(self.ctx, grid)

    def mass_history(self, grid=0):
        return L.lb_mass_history(self.ctx, grid)

    def checkpoint(self, path):
        L.lb_checkpoint(self.ctx, path)

    def restore(self, path):
        L.lb_restore(self.ctx, path)

    def close(self):
        if getattr(self, "ctx", None):
            L.lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
