"""ctypes wrapper over lb_oracle.c, the FP64 column-physics step.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function follows
the step as lb_oracle.c states it: advection (Sec. IV dynamics stand-in),
then k_c(i,j) passes of the implicit vertical solve (Fig. 1 / Fig. 4
recurrence, Sec. VI-B load array), then the compensated global sum.
"""
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_SRC = os.path.join(_HERE, "lb_oracle.c")


def build_oracle(force=False):
    """Compile lb_oracle.c (plain C, FP64, no fast-math) into _build/liborc.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _CGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
                ("r", ctypes.c_double), ("kc_mode", ctypes.c_int32),
                ("kc", ctypes.POINTER(ctypes.c_int32)),
                ("disk_x0", ctypes.c_int32), ("disk_y0", ctypes.c_int32),
                ("disk_vx", ctypes.c_int32), ("disk_vy", ctypes.c_int32),
                ("disk_r", ctypes.c_int32), ("k_in", ctypes.c_int32),
                ("k_out", ctypes.c_int32), ("dynamics", ctypes.c_int32),
                ("nu", ctypes.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_long
        P = ctypes.c_void_p
        _lib.orc_kc_field.argtypes = [ctypes.POINTER(_CGrid), i64, P]
        _lib.orc_thomas.argtypes = [i32, d, P, P, P]
        _lib.orc_advect.argtypes = [ctypes.POINTER(_CGrid), ctypes.c_int, P, P]
        _lib.orc_jacobi.argtypes = [ctypes.POINTER(_CGrid), ctypes.c_int, P, P]
        _lib.orc_sum.argtypes = [P, i64, P]
        _lib.orc_sum.restype = d
        _lib.orc_step.argtypes = [ctypes.POINTER(_CGrid), ctypes.c_int, P, P, P]
        _lib.orc_run.argtypes = [ctypes.POINTER(_CGrid), i64, i32, P, P, P]
        _lib.orc_run_window.argtypes = [ctypes.POINTER(_CGrid), i64, i64, i32, i32, i64,
                                        i32, P, P, i32]
    return _lib


@dataclass
class OracleGrid:
    """One grid: sizes, Courant numbers, diffusion number r = kappa dt / dz^2,
    and the k_c source (moving disk, or an int32 (ny, nx) array)."""
    nx: int
    ny: int
    nz: int
    cx: float = 0.5
    cy: float = 0.5
    cz: float = 0.0
    r: float = 0.1
    kc_disk: bool = True
    disk: tuple = (0, 0, 0, 0, 0)      # x0, y0, vx, vy, R (cells, cells/step)
    k_in: int = 1
    k_out: int = 1
    kc: np.ndarray = None              # (ny, nx) int32 when kc_disk is False
    dynamics: int = 0                  # 0: upwind advection; 1: weighted Jacobi sweep
    nu: float = 1.0 / 7.0              # Jacobi weight

    @classmethod
    def from_spec(cls, g, kc=None):
        return cls(g.nx, g.ny, g.nz, g.cx, g.cy, g.cz, g.r, g.kc_disk, tuple(g.disk),
                   g.k_in, g.k_out, kc, getattr(g, "dynamics", 0), getattr(g, "nu", 1.0 / 7.0))

    def _c(self):
        kc = None
        if not self.kc_disk and self.kc is not None:    # window runs bring their own
            self._kc_keep = np.ascontiguousarray(self.kc, dtype=np.int32)
            kc = self._kc_keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        x0, y0, vx, vy, R = self.disk
        return _CGrid(self.nx, self.ny, self.nz, self.cx, self.cy, self.cz, self.r,
                      1 if self.kc_disk else 0, kc, x0, y0, vx, vy, R,
                      self.k_in, self.k_out, self.dynamics, self.nu)


def _f64(q):
    return np.ascontiguousarray(q, dtype=np.float64)


def kc_field(g, t):
    """k_c(i, j, t) for every column, int32 (ny, nx)."""
    out = np.empty((g.ny, g.nx), np.int32)
    cg = g._c()
    _L().orc_kc_field(ctypes.byref(cg), t, out.ctypes.data)
    return out


def thomas(d, r):
    """One implicit vertical solve M x = d (zero-flux ends) on a 1-D column."""
    x = _f64(d).copy()
    n = x.size
    cp = np.empty(max(n, 1))
    dp = np.empty(max(n, 1))
    _L().orc_thomas(n, r, x.ctypes.data, cp.ctypes.data, dp.ctypes.data)
    return x


def advect(g, q, periodic=True):
    q = _f64(q)
    out = np.empty_like(q)
    cg = g._c()
    _L().orc_advect(ctypes.byref(cg), 1 if periodic else 0, q.ctypes.data, out.ctypes.data)
    return out


def jacobi(g, q, periodic=True):
    """One weighted Jacobi sweep of the 7-point stencil (the Sec. IV dynamics
    phase, dynamics == 1), periodic in x/y, mirror ghosts in z."""
    q = _f64(q)
    out = np.empty_like(q)
    cg = g._c()
    _L().orc_jacobi(ctypes.byref(cg), 1 if periodic else 0, q.ctypes.data, out.ctypes.data)
    return out


def step(g, q, kc, periodic=True):
    """One step (dynamics -- advection or the Jacobi sweep -- then k_c sweeps
    per column) with a given k_c array."""
    q = _f64(q)
    kc = np.ascontiguousarray(kc, dtype=np.int32)
    out = np.empty_like(q)
    cg = g._c()
    _L().orc_step(ctypes.byref(cg), 1 if periodic else 0, kc.ctypes.data,
                  q.ctypes.data, out.ctypes.data)
    return out


def run(g, q, nsteps, t0=0, kc_fields=None):
    """nsteps periodic steps from global step t0.  Returns (q, mass[nsteps]).
    kc_fields: optional (nsteps, ny, nx) int32 for array-k_c grids."""
    q = _f64(q).copy()
    mass = np.empty(max(nsteps, 1))
    kcp = None
    if kc_fields is not None:
        kc_fields = np.ascontiguousarray(kc_fields, dtype=np.int32)
        kcp = kc_fields.ctypes.data
    cg = g._c()
    _L().orc_run(ctypes.byref(cg), t0, nsteps, q.ctypes.data, mass.ctypes.data, kcp)
    return q, mass[:nsteps]


def run_window(g, q_full, i0, j0, wx, wy, nsteps, t0=0, kc_window=None):
    """Window run on columns [i0, i0+wx) x [j0, j0+wy) (periodic indices).

    Returns the (nz, wy, wx) window after nsteps; columns whose upwind
    dependence left the window are NaN.  kc_window: (wy, wx) or
    (nsteps, wy, wx) int32 for array-k_c grids.
    """
    ii = np.arange(i0, i0 + wx) % g.nx
    jj = np.arange(j0, j0 + wy) % g.ny
    w = _f64(np.asarray(q_full)[:, jj][:, :, ii]).copy()
    kcp, per_step = None, 0
    if not g.kc_disk:
        kc_window = np.ascontiguousarray(kc_window, dtype=np.int32)
        per_step = 1 if kc_window.ndim == 3 else 0
        kcp = kc_window.ctypes.data
    cg = g._c()
    _L().orc_run_window(ctypes.byref(cg), i0, j0, wx, wy, t0, nsteps, w.ctypes.data,
                        kcp, per_step)
    return w


def compensated_sum(x):
    """Neumaier-compensated FP64 sum."""
    x = _f64(x).ravel()
    return _L().orc_sum(x.ctypes.data, x.size, None)
