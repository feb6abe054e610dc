"""Shared helpers of the GPU tests: storage rounding on the CPU, oracle runs
of a grid description, normwise errors."""
import numpy as np
import torch

import oracle
from oracle import OracleGrid

_TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


class Grid:
    """A grid description accepted by Simulation and by the oracle."""

    def __init__(self, nx, ny, nz, cx=0.5, cy=0.5, cz=0.0, r=0.1, storage="f32",
                 compute="f32", kc_disk=True, disk=(0, 0, 1, 1, 3), k_in=4, k_out=1,
                 dynamics=0, nu=1.0 / 7.0, pitch=0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.pitch = pitch
        self.cx, self.cy, self.cz, self.r = cx, cy, cz, r
        self.storage, self.compute = storage, compute
        self.kc_disk, self.disk, self.k_in, self.k_out = kc_disk, tuple(disk), k_in, k_out
        self.dynamics, self.nu = dynamics, nu

    def oracle(self, kc=None):
        return OracleGrid(self.nx, self.ny, self.nz, self.cx, self.cy, self.cz, self.r,
                          self.kc_disk, self.disk, self.k_in, self.k_out, kc, self.dynamics,
                          self.nu)


def round_to_storage(q, storage):
    """The field as the storage type holds it, back in float64 (CPU rounding)."""
    t = torch.from_numpy(np.ascontiguousarray(q, dtype=np.float64))
    if storage == "f32":
        t = t.to(torch.float32)
    elif storage == "bf16":
        t = t.to(torch.float32).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def tolerance(g, nsteps):
    """Normwise bound per precision: the FP32 target 1e-5; FP64 compute 1e-12;
    BF16 storage: one rounding of relative size at most 2^-9 per stored step,
    carried through a non-expansive step operator (convex advection, M^-1
    with unit row sums and nonnegative entries).  Round-to-nearest-even makes
    the roundings unbiased, so their sum grows like sqrt(T), not T: the
    bound allows 1 + 2 sqrt(T) roundings' worth (0.030 at 50 steps, where
    the worst case T 2^-9 would be 0.098), plus the FP32 target."""
    if g.storage == "bf16":
        return (1.0 + 2.0 * nsteps ** 0.5) * 2.0 ** -9 + 1e-5
    if g.compute == "f64":
        return 1e-12
    return 1e-5


def normwise(gpu, ref):
    return float(np.abs(gpu - ref).max() / max(np.abs(ref).max(), 1e-300))


def random_field(g, seed, lo=0.2, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(g.nz, g.ny, g.nx))


def item_kc(kc, vp, item_w, item_h):
    """k_c values of each work item of VP (grid, x0, y0, w, h), in the
    kernel's item shape (lb_info.item_w / item_h): item_w x item_h tiles in
    row-major order, or (item_h == 0) runs of item_w columns of the VP in
    row-major order."""
    _, x0, y0, w, h = vp
    block = kc[y0:y0 + h, x0:x0 + w]
    if item_h == 0:
        flat = block.ravel()
        return [flat[c:c + item_w] for c in range(0, flat.size, item_w)]
    out = []
    for ty in range(0, h, item_h):
        for tx in range(0, w, item_w):
            out.append(block[ty:ty + item_h, tx:tx + item_w].ravel())
    return out


def report(name, **metrics):
    """Append measured metrics to the JSON file named by LB_REPORT (if set):
    the error and drift figures the design notes state per workload."""
    import json
    import os
    path = os.environ.get("LB_REPORT")
    if not path:
        return
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[name] = {k: (float(v) if v is not None else None) for k, v in metrics.items()}
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def mass_drift(hist, m0):
    """Largest per-step change and total change of the global sum, relative
    to the initial sum."""
    h = np.concatenate([[m0], np.asarray(hist, dtype=np.float64)])
    return float(np.abs(np.diff(h)).max() / abs(m0)), float(abs(h[-1] - m0) / abs(m0))
