"""The five synthetic workloads, with every unstated parameter fixed here.

Each workload is a list of grids plus a VP layout and a run length.  All
random draws come from SplitMix64 streams derived from the workload seed.
Names describe the workload; `get_config(name)` builds it.

  plain_fp64_64x64x32        64x64x32 FP64, 16 VPs of 16x16, 10 steps, static disk
  hotspot_fp32_512x512x64    512x512x64 FP32, 256 VPs of 32x32, 100 steps, moving disk
  lognormal_fp32_1024x1024x96  1024x1024x96 FP32, 4096 guillotine VPs (x extents on
                               8-column sectors), 200 steps, lognormal k_c re-drawn every 50 steps
  jacobi_fp32_1024x1024x96     the same with the Jacobi dynamics (7-point sweep) in place of
                               the advection
  precision_2048x2048x64     2048x2048x64, FP64/FP32/BF16 storage, FP32 compute, 50 steps
  batch64_fp32               64 grids s x s x nz, s in 64..512, nz in 32..96, FP32, rows
                             padded to multiples of 8 values in device memory
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

from .fields import gaussian_blob
from .kcfield import lognormal_kc
from .layouts import guillotine, regular_blocks
from .rng import splitmix64, subseed


@dataclass
class GridSpec:
    nx: int
    ny: int
    nz: int
    cx: float = 0.5
    cy: float = 0.5
    cz: float = 0.0
    r: float = 0.1
    storage: str = "f32"          # "f64" | "f32" | "bf16"
    compute: str = "f32"          # "f64" | "f32"
    kc_disk: bool = True          # moving-disk rule; False: caller array
    disk: Tuple[int, int, int, int, int] = (0, 0, 1, 1, 1)  # x0, y0, vx, vy, R
    k_in: int = 1
    k_out: int = 1
    center: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    sigma: float = 1.0
    noise: float = 1e-3
    seed: int = 0
    dynamics: int = 0             # 0: upwind advection; 1: weighted Jacobi sweep (Sec. IV)
    nu: float = 1.0 / 7.0         # Jacobi weight
    pitch: int = 0                # row pitch of the device buffers (0: dense rows of nx)

    def initial_field(self, dtype=np.float64):
        return gaussian_blob(self.nx, self.ny, self.nz, self.center, self.sigma,
                             self.noise, self.seed, dtype=dtype)


@dataclass
class Workload:
    name: str
    grids: List[GridSpec]
    vps: List[tuple]
    steps: int
    seed: int
    period: int = 0                      # rebalance period in steps (0: never)
    kc_epoch_steps: int = 0              # array k_c re-drawn every this many steps
    kc_params: dict = field(default_factory=dict)
    notes: str = ""

    def kc_array(self, grid, epoch):
        """k_c array of `grid` for a re-draw epoch (array-k_c workloads only)."""
        g = self.grids[grid]
        return lognormal_kc(g.nx, g.ny, subseed(self.seed, 7000 + grid), epoch,
                            **self.kc_params)

    @property
    def cells(self):
        return sum(g.nx * g.ny * g.nz for g in self.grids)


def _blob(nx, ny, nz):
    return (nx / 2.0, ny / 2.0, nz / 2.0), nx / 8.0


def plain_fp64_64x64x32():
    g = GridSpec(64, 64, 32, 0.5, 0.5, 0.0, 0.1, "f64", "f64", True,
                 (24, 40, 0, 0, 12), 8, 1, (32.0, 32.0, 16.0), 8.0, 1e-3, 1)
    return Workload("plain_fp64_64x64x32", [g], regular_blocks(64, 64, 16, 16), 10, 1,
                    notes="static disk R=12 at (24,40), k_c 8 inside, 1 outside")


def hotspot_fp32_512x512x64(storage="f32"):
    c, s = _blob(512, 512, 64)
    g = GridSpec(512, 512, 64, 0.5, 0.5, 0.0, 0.1, storage, "f32", True,
                 (128, 128, 1, 1, 64), 32, 1, c, s, 1e-3, 2)
    return Workload("hotspot_fp32_512x512x64", [g], regular_blocks(512, 512, 32, 32), 100, 2,
                    period=10, notes="disk R=64 moving (1,1)/step from (128,128), k_c 32/1")


def lognormal_fp32_1024x1024x96():
    c, s = _blob(1024, 1024, 96)
    g = GridSpec(1024, 1024, 96, 0.5, 0.5, 0.0, 0.1, "f32", "f32", False,
                 (0, 0, 0, 0, 0), 1, 1, c, s, 1e-3, 3)
    # x extents on multiples of 8 columns: every VP row segment starts on a
    # 32-byte sector (FP32), so no sector is shared by two VPs
    vps = guillotine(1024, 1024, 4096, 8, subseed(3, 11), x_align=8)
    return Workload("lognormal_fp32_1024x1024x96", [g], vps, 200, 3, period=10,
                    kc_epoch_steps=50,
                    notes="guillotine VPs, lognormal k_c (mu=1, smoothed sigma 4) in 1..64")


def jacobi_fp32_1024x1024x96():
    """The lognormal workload with the Sec. IV dynamics in its Jacobi form:
    one weighted 7-point Jacobi sweep (nu = 1/7) per step in place of the
    advection; same grid, VPs, k_c arrays and re-draws."""
    w = lognormal_fp32_1024x1024x96()
    g = w.grids[0]
    g.cx = g.cy = g.cz = 0.0
    g.dynamics, g.nu = 1, 1.0 / 7.0
    w.name = "jacobi_fp32_1024x1024x96"
    w.notes = "Jacobi dynamics (nu 1/7); " + w.notes
    return w


def precision_2048x2048x64(storage="f32"):
    c, s = _blob(2048, 2048, 64)
    g = GridSpec(2048, 2048, 64, 0.5, 0.5, 0.0, 0.1, storage, "f32", True,
                 (512, 512, 1, 1, 256), 32, 1, c, s, 1e-3, 4)
    return Workload("precision_2048x2048x64_" + storage, [g],
                    regular_blocks(2048, 2048, 64, 64), 50, 4, period=10,
                    notes="disk R=256 moving (1,1)/step from (512,512), k_c 32/1")


def batch64_fp32(ngrids=64, pad=True):
    """64 grids of side s in 64..512: the device buffers pad each row to a
    multiple of 8 FP32 values (pad=True), so that every row, and every VP
    row segment (VPs start on multiples of 32 columns), begins on a 32-byte
    sector; the fields themselves are s x s x nz."""
    seed = 5
    grids, vps = [], []
    rs = subseed(seed, 21)
    for gi in range(ngrids):
        side = 64 + int(splitmix64(rs, 6 * gi) % np.uint64(512 - 64 + 1))
        nz = 32 + int(splitmix64(rs, 6 * gi + 1) % np.uint64(96 - 32 + 1))
        kin = 2 + int(splitmix64(rs, 6 * gi + 2) % np.uint64(48 - 2 + 1))
        x0 = int(splitmix64(rs, 6 * gi + 3) % np.uint64(side))
        y0 = int(splitmix64(rs, 6 * gi + 4) % np.uint64(side))
        c, s = _blob(side, side, nz)
        grids.append(GridSpec(side, side, nz, 0.5, 0.5, 0.0, 0.1, "f32", "f32", True,
                              (x0, y0, 1, 1, side // 8), kin, 1, c, s, 1e-3,
                              subseed(seed, 100 + gi), pitch=(side + 7) // 8 * 8 if pad else 0))
        vps += regular_blocks(side, side, 32, 32, grid=gi)
    return Workload("batch64_fp32", grids, vps, 50, seed, period=10,
                    notes="64 grids, side U{64..512}, nz U{32..96}, k_in U{2..48}")


CONFIGS = {
    "plain_fp64_64x64x32": plain_fp64_64x64x32,
    "hotspot_fp32_512x512x64": hotspot_fp32_512x512x64,
    "lognormal_fp32_1024x1024x96": lognormal_fp32_1024x1024x96,
    "jacobi_fp32_1024x1024x96": jacobi_fp32_1024x1024x96,
    "precision_2048x2048x64": precision_2048x2048x64,
    "batch64_fp32": batch64_fp32,
}


def get_config(name, **kw):
    return CONFIGS[name](**kw)
