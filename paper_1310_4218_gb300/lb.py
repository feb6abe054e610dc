"""ctypes binding of liblb.so: the C ABI of include/lb.h under the same names.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Device buffers are passed as integers (torch `data_ptr()`),
host buffers as numpy arrays.  A non-OK status raises LBError carrying the
library's lb_last_error text.  If the library is missing the import fails:
there is no fallback.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "liblb.so")

(LB_OK, LB_EINVAL, LB_ECUDA, LB_ETIMEOUT, LB_ENUMERIC, LB_ESTATE, LB_ENORESIDENT, LB_EIO,
 LB_EKCRANGE) = range(9)
LB_KC_MAX = 1024
LB_F64, LB_F32, LB_BF16 = 0, 1, 2
(LB_STATIC, LB_GREEDY, LB_REFINE_SWAP, LB_ATOMIC_QUEUE, LB_AUTO, LB_GREEDY_SPATIAL,
 LB_AUTO_SPATIAL, LB_GREEDY_BLOCKED) = range(8)

STATUS_NAMES = {0: "LB_OK", 1: "LB_EINVAL", 2: "LB_ECUDA", 3: "LB_ETIMEOUT", 4: "LB_ENUMERIC",
                5: "LB_ESTATE", 6: "LB_ENORESIDENT", 7: "LB_EIO", 8: "LB_EKCRANGE"}
DTYPES = {"f64": LB_F64, "f32": LB_F32, "bf16": LB_BF16}
STRATEGIES = {"static": LB_STATIC, "greedy": LB_GREEDY, "refine_swap": LB_REFINE_SWAP,
              "queue": LB_ATOMIC_QUEUE, "auto": LB_AUTO, "greedy_spatial": LB_GREEDY_SPATIAL,
              "auto_spatial": LB_AUTO_SPATIAL, "greedy_blocked": LB_GREEDY_BLOCKED}


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class lb_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
                ("r", ctypes.c_double), ("storage", ctypes.c_int32), ("compute", ctypes.c_int32),
                ("q0", ctypes.c_void_p), ("q1", ctypes.c_void_p), ("kc", ctypes.c_void_p),
                ("kc_disk", ctypes.c_int32), ("disk_x0", ctypes.c_int32),
                ("disk_y0", ctypes.c_int32), ("disk_vx", ctypes.c_int32),
                ("disk_vy", ctypes.c_int32), ("disk_r", ctypes.c_int32),
                ("k_in", ctypes.c_int32), ("k_out", ctypes.c_int32),
                ("dynamics", ctypes.c_int32), ("pitch", ctypes.c_int32), ("nu", ctypes.c_double)]


class lb_vp(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("x0", ctypes.c_int32), ("y0", ctypes.c_int32),
                ("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class lb_options(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("queue_order", ctypes.c_int32),
                ("mass_every", ctypes.c_int32), ("device_balancer", ctypes.c_int32),
                ("ema_alpha", ctypes.c_double), ("refine_tol", ctypes.c_double),
                ("barrier_timeout_ns", ctypes.c_int64), ("threads_hint", ctypes.c_int32),
                ("steal", ctypes.c_int32), ("predict_kc", ctypes.c_int32),
                ("staged_loads", ctypes.c_int32), ("dataflow", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class lb_info(ctypes.Structure):
    _fields_ = [("nprocs", ctypes.c_int32), ("nsm", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("max_ctas_per_sm", ctypes.c_int32),
                ("nz_variant", ctypes.c_int32), ("exact_nz", ctypes.c_int32),
                ("step", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("strategy", ctypes.c_int32), ("regs_per_thread", ctypes.c_int32),
                ("item_w", ctypes.c_int32), ("item_h", ctypes.c_int32),
                ("staged_slots", ctypes.c_int32), ("dataflow", ctypes.c_int32)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIG = {
    "lb_default_options": (None, [ctypes.POINTER(lb_options)]),
    "lb_create": (_I32, [ctypes.POINTER(lb_grid_desc), _I32, ctypes.POINTER(lb_vp), _I32,
                         ctypes.POINTER(lb_options), _P, ctypes.POINTER(_P)]),
    "lb_step": (_I32, [_P, _I32]),
    "lb_measure_loads": (_I32, [_P, _P, _P, _P]),
    "lb_rebalance": (_I32, [_P, _I32, _P, _P]),
    "lb_plan": (_I32, [_I32, _P, _I32, _I32, _P, ctypes.c_double, _P, _P, _P]),
    "lb_set_costs": (_I32, [_P, _P]),
    "lb_get_assignment": (_I32, [_P, _P, _P]),
    "lb_set_assignment": (_I32, [_P, _P]),
    "lb_set_kc": (_I32, [_P, _I32, _P]),
    "lb_mass": (_I32, [_P, _I32, _P, _P]),
    "lb_mass_history": (_I32, [_P, _I32, _P, _I32, _P]),
    "lb_work_done": (_I32, [_P, _P, _P]),
    "lb_current_field": (_I32, [_P, _I32, ctypes.POINTER(_P)]),
    "lb_sync": (_I32, [_P]),
    "lb_graph_create": (_I32, [_P, _I32, ctypes.POINTER(_P)]),
    "lb_graph_launch": (_I32, [_P, _P]),
    "lb_graph_destroy": (_I32, [_P, _P]),
    "lb_checkpoint": (_I32, [_P, ctypes.c_char_p]),
    "lb_restore": (_I32, [_P, ctypes.c_char_p]),
    "lb_get_info": (_I32, [_P, ctypes.POINTER(lb_info)]),
    "lb_last_error": (ctypes.c_char_p, [_P]),
    "lb_destroy": (None, [_P]),
    "lb_device_measure": (_I32, [_P]),
    "lb_device_rebalance": (_I32, [_P, _I32]),
    "lb_device_rebalance_if": (_I32, [_P, _I32, ctypes.c_double]),
    "lb_get_costs": (_I32, [_P, _P, _P]),
    "lb_balance_history": (_I32, [_P, _P, _I32, _P]),
    "lb_graph_create_periods": (_I32, [_P, _I32, _I32, _I32, ctypes.c_double,
                                       ctypes.POINTER(_P)]),
    "lb_step_noalloc": (_I32, [ctypes.POINTER(lb_grid_desc), ctypes.POINTER(lb_vp), _I32,
                               _P, ctypes.c_int64, _I32, _P, _P]),
    "lb_set_owned": (_I32, [_P, _P]),
    "lb_step_serial": (_I32, [_P, _I32]),
    "lb_pack_columns": (_I32, [_P, _I32, _P, _I32, _P]),
    "lb_unpack_columns": (_I32, [_P, _I32, _P, _I32, _P]),
}
EXPORTED = tuple(_SIG)

_lib = None


def load_library(path=None):
    """Load liblb.so (built by paper_1310_4218_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError("liblb.so not built (%s); run __graft_entry__.build()" % p)
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIG.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(status, ctx=None):
    if status != LB_OK:
        msg = load_library().lb_last_error(ctx)
        raise LBError(status, msg.decode() if msg else "")


def _ptr(a):
    return None if a is None else a.ctypes.data


def lb_default_options():
    o = lb_options()
    load_library().lb_default_options(ctypes.byref(o))
    return o


def lb_create(grids, vps, options=None, stream=0):
    """grids: list of lb_grid_desc; vps: list of (grid, x0, y0, w, h);
    stream: cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream)."""
    L = load_library()
    ga = (lb_grid_desc * len(grids))(*grids)
    va = (lb_vp * len(vps))(*[lb_vp(*map(int, v)) for v in vps])
    out = _P()
    st = L.lb_create(ga, len(grids), va, len(vps),
                     ctypes.byref(options) if options is not None else None,
                     _P(stream or 0), ctypes.byref(out))
    _check(st, None)
    return out.value


def lb_step(ctx, nsteps):
    _check(load_library().lb_step(ctx, int(nsteps)), ctx)


def lb_measure_loads(ctx, nvps, nsm=None):
    """Returns (vp_cost_ns[nvps], sm_busy_ns[nsm])."""
    info = lb_get_info(ctx)
    vc = np.zeros(nvps, np.float64)
    sb = np.zeros(info.nsm, np.float64)
    n = ctypes.c_int32(0)
    _check(load_library().lb_measure_loads(ctx, _ptr(vc), _ptr(sb), ctypes.addressof(n)), ctx)
    return vc, sb[:n.value]


def lb_rebalance(ctx, strategy):
    """Returns (migrations, predicted max/mean)."""
    m = ctypes.c_int32(0)
    p = ctypes.c_double(0.0)
    s = STRATEGIES.get(strategy, strategy)
    _check(load_library().lb_rebalance(ctx, int(s), ctypes.addressof(m), ctypes.addressof(p)), ctx)
    return m.value, p.value


def lb_plan(strategy, costs, nprocs, current=None, refine_tol=0.05):
    """Host-only balancer: returns (assignment, migrations, predicted max/mean)."""
    c = np.ascontiguousarray(costs, dtype=np.float64)
    cur = None if current is None else np.ascontiguousarray(current, dtype=np.int32)
    out = np.zeros(c.size, np.int32)
    m = ctypes.c_int32(0)
    p = ctypes.c_double(0.0)
    s = STRATEGIES.get(strategy, strategy)
    _check(load_library().lb_plan(int(s), _ptr(c), c.size, int(nprocs), _ptr(cur),
                                  float(refine_tol), _ptr(out), ctypes.addressof(m),
                                  ctypes.addressof(p)))
    return out, m.value, p.value


def lb_set_costs(ctx, costs):
    c = np.ascontiguousarray(costs, dtype=np.float64)
    _check(load_library().lb_set_costs(ctx, _ptr(c)), ctx)


def lb_get_assignment(ctx, nvps):
    a = np.zeros(nvps, np.int32)
    n = ctypes.c_int32(0)
    _check(load_library().lb_get_assignment(ctx, _ptr(a), ctypes.addressof(n)), ctx)
    return a, n.value


def lb_set_assignment(ctx, assign):
    a = np.ascontiguousarray(assign, dtype=np.int32)
    _check(load_library().lb_set_assignment(ctx, _ptr(a)), ctx)


def lb_set_kc(ctx, grid, dev_kc_ptr):
    _check(load_library().lb_set_kc(ctx, int(grid), _P(dev_kc_ptr)), ctx)


def lb_mass(ctx, grid=0):
    s = ctypes.c_double(0.0)
    c = ctypes.c_double(0.0)
    _check(load_library().lb_mass(ctx, int(grid), ctypes.addressof(s), ctypes.addressof(c)), ctx)
    return s.value, c.value


def lb_mass_history(ctx, grid=0, max_entries=1024):
    buf = np.zeros(max_entries, np.float64)
    n = ctypes.c_int32(0)
    _check(load_library().lb_mass_history(ctx, int(grid), _ptr(buf), int(max_entries),
                                          ctypes.addressof(n)), ctx)
    return buf[:n.value]


def lb_work_done(ctx):
    """(cell_sweeps, cell_steps) performed since lb_create, counted on the device."""
    a = ctypes.c_int64(0)
    b = ctypes.c_int64(0)
    _check(load_library().lb_work_done(ctx, ctypes.addressof(a), ctypes.addressof(b)), ctx)
    return a.value, b.value


def lb_current_field(ctx, grid=0):
    p = _P()
    _check(load_library().lb_current_field(ctx, int(grid), ctypes.byref(p)), ctx)
    return p.value


def lb_graph_create(ctx, nsteps):
    """Executable CUDA graph of one nsteps-step launch (handle as int)."""
    g = _P()
    _check(load_library().lb_graph_create(ctx, int(nsteps), ctypes.byref(g)), ctx)
    return g.value


def lb_graph_launch(ctx, graph):
    _check(load_library().lb_graph_launch(ctx, _P(graph)), ctx)


def lb_graph_destroy(ctx, graph):
    _check(load_library().lb_graph_destroy(ctx, _P(graph)), ctx)


def lb_device_measure(ctx):
    _check(load_library().lb_device_measure(ctx), ctx)


def lb_device_rebalance(ctx, strategy):
    s = STRATEGIES.get(strategy, strategy)
    _check(load_library().lb_device_rebalance(ctx, int(s)), ctx)


def lb_device_rebalance_if(ctx, strategy, threshold):
    s = STRATEGIES.get(strategy, strategy)
    _check(load_library().lb_device_rebalance_if(ctx, int(s), float(threshold)), ctx)


def lb_get_costs(ctx, nvps):
    """(cost average, last measurement) per VP, ns per step."""
    a = np.zeros(nvps, np.float64)
    b = np.zeros(nvps, np.float64)
    _check(load_library().lb_get_costs(ctx, _ptr(a), _ptr(b)), ctx)
    return a, b


BALANCE_HISTORY_COLUMNS = ("step", "strategy", "migrations", "predicted_max_over_mean",
                           "sm_max_over_mean", "granularity_floor", "refine_iterations", "kept")


def lb_balance_history(ctx, max_rows=1024):
    """Device rebalances, oldest first: float64 array [n, 8] with the
    columns of BALANCE_HISTORY_COLUMNS."""
    buf = np.zeros((max_rows, 8), np.float64)
    n = ctypes.c_int32(0)
    _check(load_library().lb_balance_history(ctx, _ptr(buf), int(max_rows),
                                             ctypes.addressof(n)), ctx)
    return buf[:n.value]


def lb_graph_create_periods(ctx, nsteps, strategy, nperiods, threshold=0.0):
    """Executable CUDA graph of nperiods x (nsteps steps, device measurement,
    device rebalance within threshold)."""
    g = _P()
    s = STRATEGIES.get(strategy, strategy)
    _check(load_library().lb_graph_create_periods(ctx, int(nsteps), int(s), int(nperiods),
                                                  float(threshold), ctypes.byref(g)), ctx)
    return g.value


def lb_sync(ctx):
    _check(load_library().lb_sync(ctx), ctx)


def lb_checkpoint(ctx, path):
    _check(load_library().lb_checkpoint(ctx, os.fsencode(path)), ctx)


def lb_restore(ctx, path):
    _check(load_library().lb_restore(ctx, os.fsencode(path)), ctx)


def lb_get_info(ctx):
    i = lb_info()
    _check(load_library().lb_get_info(ctx, ctypes.byref(i)), ctx)
    return i


def lb_last_error(ctx=None):
    m = load_library().lb_last_error(ctx)
    return m.decode() if m else ""


def lb_destroy(ctx):
    if ctx:
        load_library().lb_destroy(ctx)


def lb_step_noalloc(grid, vps, t0, nsteps, stream=0, want_mass=True, options=None):
    """nsteps steps of one grid with no memory allocation in the library (a
    fixed device array inside liblb.so holds every table); returns the global
    sum after the last step, or None.  options: an lb_options or None (the
    defaults)."""
    L = load_library()
    va = (lb_vp * len(vps))(*[lb_vp(*map(int, v)) for v in vps])
    m = ctypes.c_double(0.0)
    st = L.lb_step_noalloc(ctypes.byref(grid), va, len(vps),
                           ctypes.byref(options) if options is not None else None, int(t0),
                           int(nsteps), _P(stream or 0), ctypes.addressof(m) if want_mass else None)
    _check(st, None)
    return m.value if want_mass else None


def lb_set_owned(ctx, owned):
    """Run only the VPs whose entry of owned (length nvps, 0/1) is 1."""
    a = np.ascontiguousarray(owned, dtype=np.uint8)
    _check(load_library().lb_set_owned(ctx, _ptr(a)), ctx)


def lb_pack_columns(ctx, grid, cells_ptr, n, buf_ptr):
    """Enqueue a copy of n columns (device int32 indices at cells_ptr) of the
    current field into the device buffer at buf_ptr (level-major)."""
    _check(load_library().lb_pack_columns(ctx, int(grid), _P(cells_ptr or 0), int(n),
                                          _P(buf_ptr or 0)), ctx)


def lb_unpack_columns(ctx, grid, cells_ptr, n, buf_ptr):
    """Enqueue a copy of a level-major device buffer into n columns of the
    current field."""
    _check(load_library().lb_unpack_columns(ctx, int(grid), _P(cells_ptr or 0), int(n),
                                            _P(buf_ptr or 0)), ctx)


def lb_step_serial(ctx, nsteps):
    """nsteps steps with one working warp per processor (serialized
    measurement: costs free of interference from co-running warps)."""
    _check(load_library().lb_step_serial(ctx, int(nsteps)), ctx)
