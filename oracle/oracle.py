"""ctypes front end of the FP64 oracle in ``cue_oracle.c``.

Test infrastructure only (see the package docstring).  Every function takes
and returns numpy arrays; fields are shaped (ny, nx) in 2D and (nz, ny, nx) in
3D (C order, x fastest); cone state is structure-of-arrays, pos/dir shaped
(dim, n), active shaped (n,) uint8.
"""
from __future__ import annotations

import ctypes as ct
import math
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cue_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Grid(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int),
                ("h", ct.c_double), ("D", ct.c_double), ("lam", ct.c_double), ("dt", ct.c_double)]


class _Cone(ct.Structure):
    _fields_ = [("w_prev", ct.c_double), ("w_grad", ct.c_double), ("w_noise", ct.c_double),
                ("step_len", ct.c_double), ("stop_radius", ct.c_double), ("grad_eps", ct.c_double),
                ("wall_mode", ct.c_int), ("seed", ct.c_uint64), ("steer", ct.c_int),
                ("snr_gain", ct.c_double), ("snr_width", ct.c_double), ("snr_kd", ct.c_double),
                ("snr_cmin", ct.c_double), ("snr_cmax", ct.c_double), ("snr_turn", ct.c_double)]


@dataclasses.dataclass
class Grid:
    """Grid and field physics: node i of an axis sits at x = i*h."""
    dim: int
    nx: int
    ny: int
    nz: int = 1
    h: float = 1.0
    D: float = 1.0
    lam: float = 0.0
    dt: float = 0.2

    def _c(self) -> _Grid:
        return _Grid(self.dim, self.nx, self.ny, self.nz if self.dim == 3 else 1,
                     self.h, self.D, self.lam, self.dt)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.dim == 3 else (self.ny, self.nx)

    @property
    def extents(self):
        return (self.nx, self.ny, self.nz)[: self.dim]


@dataclasses.dataclass
class Cone:
    """Growth-cone steering parameters."""
    w_prev: float = 0.5
    w_grad: float = 0.4
    w_noise: float = 0.1
    step_len: float = 0.5
    stop_radius: float = 0.0
    grad_eps: float = 1e-15
    wall_mode: int = 0
    seed: int = 0
    # SNR turn rule (Sec. 3.5, Eq. 5; 2D): steer = 1 turns by snr_turn right / left by the
    # sign of a draw from N(SNR, 1) while C(p) lies in [snr_cmin, snr_cmax]
    steer: int = 0
    snr_gain: float = 1.0
    snr_width: float = 1.0
    snr_kd: float = 1.0
    snr_cmin: float = 0.0
    snr_cmax: float = float("inf")
    snr_turn: float = math.pi / 30

    def _c(self) -> _Cone:
        return _Cone(self.w_prev, self.w_grad, self.w_noise, self.step_len, self.stop_radius,
                     self.grad_eps, self.wall_mode, self.seed & 0xFFFFFFFFFFFFFFFF, self.steer,
                     self.snr_gain, self.snr_width, self.snr_kd, self.snr_cmin,
                     min(self.snr_cmax, 1.7976931348623157e308), self.snr_turn)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, FP contraction off) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP only splits the field's node loop across threads when asked to
        # (set_threads); without it the pragma is ignored and the library is the same
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            P = ct.c_void_p
            lib.orc_philox_many.argtypes = [ct.c_int, P, P, P]
            lib.orc_noise_many.argtypes = [ct.c_uint64, ct.c_int, P, P, ct.c_int, P]
            lib.orc_node_gradient.argtypes = [ct.POINTER(_Grid), P, ct.c_int, ct.c_int, ct.c_int, P]
            lib.orc_gradient_many.argtypes = [ct.POINTER(_Grid), P, ct.c_int, P, P]
            lib.orc_field_step.argtypes = [ct.POINTER(_Grid), P, P, P, P, ct.c_int, P]
            lib.orc_cone_step.argtypes = [ct.POINTER(_Grid), ct.POINTER(_Cone), P, ct.c_uint32,
                                          ct.c_int, P, P, P, P, ct.c_int]
            lib.orc_run.argtypes = [ct.POINTER(_Grid), ct.POINTER(_Cone), P, P, ct.c_uint32,
                                    ct.c_int, P, P, ct.c_int, P, ct.c_int, P, P, P]
            lib.orc_adjoint.argtypes = [ct.POINTER(_Grid), ct.POINTER(_Cone), P, P, P, ct.c_int, P, ct.c_int,
                                        P, P, P, ct.c_int, P, P, P, P, P, P, P, P, ct.c_int]
            lib.orc_adjoint.restype = ct.c_double
            lib.orc_adjoint_from_states.argtypes = [ct.POINTER(_Grid), ct.POINTER(_Cone), P, ct.c_int, ct.c_int, P,
                                                    ct.c_int, P, P, P, P, P, P, P, P]
            lib.orc_adjoint_from_states.restype = ct.c_double
            lib.orc_bin_points.argtypes = [ct.c_int, ct.c_int, P, ct.c_double, P, P, P, P, P]
            lib.orc_connect.argtypes = [ct.c_int, ct.c_int, P, P, P, ct.c_int, P, ct.c_double, ct.c_int, P, P]
            lib.orc_connect.restype = ct.c_int
            lib.orc_csr.argtypes = [ct.c_int, ct.c_int, P, P, P, P]
            lib.orc_csr.restype = ct.c_int
            lib.orc_bfs.argtypes = [ct.c_int, P, P, ct.c_int, P]
            lib.orc_set_threads.argtypes = [ct.c_int]
            lib.orc_field_window.argtypes = [ct.POINTER(_Grid), P, ct.c_int64, ct.c_int64, ct.c_int64, ct.c_int,
                                             ct.c_int, ct.c_int, P, P, ct.c_int, P]
            lib.orc_openmp.restype = ct.c_int
            lib.orc_value_at.argtypes = [ct.POINTER(_Grid), P, P]
            lib.orc_value_at.restype = ct.c_double
            lib.orc_snr.argtypes = [ct.POINTER(_Cone), ct.c_double, P, P]
            lib.orc_snr.restype = ct.c_double
            lib.orc_endpoint_loss.argtypes = [ct.POINTER(_Grid), ct.POINTER(_Cone), P, P, P, ct.c_int, P,
                                              ct.c_int, P, P, P, ct.c_int]
            lib.orc_endpoint_loss.restype = ct.c_double
            for f in ("orc_philox_many", "orc_noise_many", "orc_node_gradient",
                      "orc_gradient_many", "orc_field_step", "orc_cone_step", "orc_run"):
                getattr(lib, f).restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _src(src_cell, src_emit):
    cell = np.ascontiguousarray(np.asarray(src_cell, dtype=np.int32).reshape(-1))
    emit = None if src_emit is None else _f64(np.asarray(src_emit).reshape(-1))
    return cell, emit


def philox4x32_10(ctr, key):
    """Philox-4x32-10 of counters ``ctr`` (n,4) under keys ``key`` (n,2) -> (n,4) uint32."""
    ctr = np.ascontiguousarray(np.atleast_2d(ctr), dtype=np.uint32)
    key = np.ascontiguousarray(np.atleast_2d(key), dtype=np.uint32)
    key = np.ascontiguousarray(np.broadcast_to(key, (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    _load().orc_philox_many(ctr.shape[0], _ptr(ctr), _ptr(key), _ptr(out))
    return out


def noise(seed, axon, step, dim):
    """Box-Muller Gaussian vectors for cones ``axon`` at steps ``step`` -> (n,3) (unused tail 0)."""
    axon = np.ascontiguousarray(np.atleast_1d(axon), dtype=np.uint32)
    step = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(step), axon.shape), dtype=np.uint32)
    out = np.zeros((axon.shape[0], 3))
    _load().orc_noise_many(int(seed) & 0xFFFFFFFFFFFFFFFF, axon.shape[0], _ptr(axon), _ptr(step),
                           dim, _ptr(out))
    return out


def node_gradient(grid: Grid, C, i, j, k=0):
    C = _f64(C)
    out = np.zeros(3)
    g = grid._c()
    _load().orc_node_gradient(ct.byref(g), _ptr(C), i, j, k, _ptr(out))
    return out


def value_at(grid: Grid, C, p):
    """Bilinear cue value at 2D points ``p`` (n, 2) -> (n,)."""
    C = _f64(C)
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    out = np.empty(p.shape[0])
    g = grid._c()
    L = _load()
    for i in range(p.shape[0]):
        q = (ct.c_double * 3)(p[i, 0], p[i, 1], 0.0)
        out[i] = L.orc_value_at(ct.byref(g), _ptr(C), q)
    return out


def snr(cone: Cone, Cp, g, d):
    """Eq. 5 for one cone: cue value Cp, gradient g (2,), direction d (2,)."""
    gg = (ct.c_double * 2)(float(g[0]), float(g[1]))
    dd = (ct.c_double * 2)(float(d[0]), float(d[1]))
    c = cone._c()
    return float(_load().orc_snr(ct.byref(c), float(Cp), gg, dd))


def gradient_at(grid: Grid, C, p):
    """Interpolated gradient at points ``p`` (n, dim) -> (n, 3)."""
    C = _f64(C)
    p = np.atleast_2d(np.asarray(p, dtype=np.float64))
    pp = np.zeros((p.shape[0], 3))
    pp[:, : p.shape[1]] = p
    out = np.zeros((p.shape[0], 3))
    g = grid._c()
    _load().orc_gradient_many(ct.byref(g), _ptr(C), p.shape[0], _ptr(pp), _ptr(out))
    return out


def set_threads(n: int) -> int:
    """Threads for the field's node loop (rows are independent: results do not depend on
    the count); returns the count in effect (1 where the library has no OpenMP)."""
    lib = _load()
    n = max(1, int(n)) if lib.orc_openmp() else 1
    lib.orc_set_threads(n)
    return n


def field_step(grid: Grid, C, src_cell=(), src_emit=(), src_map=None):
    """One explicit field step; returns C^{n+1} (float64, same shape as C)."""
    C = _f64(C)
    out = np.empty_like(C)
    cell, emit = _src(src_cell, src_emit)
    smap = None if src_map is None else _f64(src_map)
    g = grid._c()
    _load().orc_field_step(ct.byref(g), _ptr(C), _ptr(out), _ptr(cell), _ptr(emit),
                           cell.shape[0], _ptr(smap))
    return out


def field_window(grid: Grid, Wp, origin, src_cell=(), src_emit=()):
    """C' on a window of a (possibly huge) grid from the window's input values grown by one
    node on every side (``Wp``: shape (wy + 2, wx + 2) in 2D, (wz + 2, wy + 2, wx + 2) in 3D;
    entries outside the grid are ignored); ``origin`` = the window's first node (x, y[, z]).
    Point sources inside the window are added; no rate map."""
    lib = _load()
    Wp = _f64(Wp)
    if grid.dim == 2:
        wy, wx = Wp.shape[0] - 2, Wp.shape[1] - 2
        wz, (ox, oy), oz = 1, origin, 0
    else:
        wz, wy, wx = Wp.shape[0] - 2, Wp.shape[1] - 2, Wp.shape[2] - 2
        ox, oy, oz = origin
    out = np.zeros((wz, wy, wx) if grid.dim == 3 else (wy, wx), np.float64)
    cells = np.ascontiguousarray(np.asarray(src_cell, np.int64).reshape(-1))
    emit = _f64(np.asarray(src_emit, np.float64).reshape(-1))
    lib.orc_field_window(ct.byref(grid._c()), _ptr(Wp), int(ox), int(oy), int(oz), wx, wy, wz,
                         _ptr(cells) if cells.size else None, _ptr(emit) if emit.size else None, int(cells.size),
                         _ptr(out))
    return out


def cone_step(grid: Grid, cone: Cone, C, step, pos, dir, active, src_cell=()):
    """One cone step on field C at step index ``step``; returns new (pos, dir, active)."""
    C = _f64(C)
    pos = _f64(pos).copy()
    dirs = _f64(dir).copy()
    act = np.ascontiguousarray(active, dtype=np.uint8).copy()
    cell, _ = _src(src_cell, None)
    g, c = grid._c(), cone._c()
    _load().orc_cone_step(ct.byref(g), ct.byref(c), _ptr(C), int(step), act.shape[0],
                          _ptr(pos), _ptr(dirs), _ptr(act), _ptr(cell), cell.shape[0])
    return pos, dirs, act


def run(grid: Grid, cone: Cone, C, step0, nsteps, src_cell=(), src_emit=(), src_map=None,
        pos=None, dir=None, active=None):
    """``nsteps`` coupled steps from step index ``step0``: cones on C^n, then C^n -> C^{n+1}.

    Returns (C, pos, dir, active) as new arrays."""
    C = _f64(C).copy()
    work = np.empty_like(C)
    cell, emit = _src(src_cell, src_emit)
    smap = None if src_map is None else _f64(src_map)
    if pos is None:
        n = 0
        pos = np.zeros((grid.dim, 0))
        dirs = np.zeros((grid.dim, 0))
        act = np.zeros(0, np.uint8)
    else:
        pos = _f64(pos).copy()
        dirs = _f64(dir).copy()
        act = np.ascontiguousarray(active, dtype=np.uint8).copy()
        n = act.shape[0]
    g, c = grid._c(), cone._c()
    _load().orc_run(ct.byref(g), ct.byref(c), _ptr(C), _ptr(work), int(step0), int(nsteps),
                    _ptr(cell), _ptr(emit), cell.shape[0], _ptr(smap), n,
                    _ptr(pos), _ptr(dirs), _ptr(act))
    return C, pos, dirs, act


def endpoint_loss(grid: Grid, cone: Cone, C0, src_cell, src_emit, src_map, pos, dir, targets, nsteps):
    """Forward loss (1/n) sum_a |p_a^T - t_a|^2 of a clamp-mode run."""
    C0 = _f64(C0)
    cell, emit = _src(src_cell, src_emit)
    smap = None if src_map is None else _f64(src_map)
    pos, dirs, tg = _f64(pos), _f64(dir), _f64(targets)
    g, c = grid._c(), cone._c()
    return float(_load().orc_endpoint_loss(ct.byref(g), ct.byref(c), _ptr(C0), _ptr(cell), _ptr(emit),
                                           cell.shape[0], _ptr(smap), pos.shape[1], _ptr(pos), _ptr(dirs),
                                           _ptr(tg), int(nsteps)))


def adjoint(grid: Grid, cone: Cone, C0, src_cell, src_emit, src_map, pos, dir, targets, nsteps,
            state_binary32=False):
    """FP64 adjoint of endpoint_loss: returns (loss, dL/dD, dL/dlambda, dL/de (n_src,),
    dL/dM (field-shaped)).  Stores every state: small problems only.

    ``state_binary32`` rounds each stored forward state to binary32 (a measuring knob for
    the tests: how far single-precision storage alone moves the gradients)."""
    C0 = _f64(C0)
    cell, emit = _src(src_cell, src_emit)
    smap = _f64(np.zeros(C0.shape) if src_map is None else src_map)
    pos, dirs, tg = _f64(pos), _f64(dir), _f64(targets)
    n = pos.shape[1]
    nn = C0.size
    T = int(nsteps)
    Cs = np.empty((T + 1) * nn)
    Ps = np.empty((T + 1) * pos.size)
    Ds = np.empty((T + 1) * pos.size)
    work = np.zeros(((n + 15) // 16) * 16 + 3 * nn * 8, dtype=np.uint8)
    gD, gl = ct.c_double(), ct.c_double()
    gsrc = np.zeros(cell.shape[0])
    gmap = np.zeros(C0.shape)
    g, c = grid._c(), cone._c()
    loss = _load().orc_adjoint(ct.byref(g), ct.byref(c), _ptr(C0), _ptr(cell), _ptr(emit), cell.shape[0],
                               _ptr(smap), n, _ptr(pos), _ptr(dirs), _ptr(tg), T, ct.byref(gD), ct.byref(gl),
                               _ptr(gsrc), _ptr(gmap), _ptr(Cs), _ptr(Ps), _ptr(Ds), _ptr(work),
                               1 if state_binary32 else 0)
    return float(loss), gD.value, gl.value, gsrc, gmap


def adjoint_from_states(grid: Grid, cone: Cone, src_cell, targets, C_states, pos_states, dir_states):
    """The oracle's backward pass alone over given forward states: ``C_states`` (T + 1,
    *field shape), ``pos_states`` / ``dir_states`` (T + 1, dim, n).  Returns (loss, dL/dD,
    dL/dlambda, dL/de (n_src,), dL/dM (field-shaped)) as :func:`adjoint` does.  Fed the
    states of another program's forward run it gives the gradients that program's backward
    pass must produce from exactly those states."""
    Cs = _f64(C_states)
    Ps, Ds, tg = _f64(pos_states), _f64(dir_states), _f64(targets)
    T = Cs.shape[0] - 1
    if T < 0 or Ps.shape[0] != T + 1 or Ds.shape[0] != T + 1:
        raise ValueError("states: T + 1 fields, positions and directions")
    n = Ps.shape[2]
    cell = _i32(src_cell)
    nn = Cs[0].size
    work = np.zeros(3 * nn)
    gD, gl = ct.c_double(), ct.c_double()
    gsrc = np.zeros(cell.shape[0])
    gmap = np.zeros(Cs.shape[1:])
    g, c = grid._c(), cone._c()
    loss = _load().orc_adjoint_from_states(ct.byref(g), ct.byref(c), _ptr(cell), cell.shape[0], n, _ptr(tg), T,
                                           _ptr(Cs), _ptr(Ps), _ptr(Ds), ct.byref(gD), ct.byref(gl), _ptr(gsrc),
                                           _ptr(gmap), _ptr(work))
    return float(loss), gD.value, gl.value, gsrc, gmap


# ------------------------------------------------------------------ connectivity
def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def bin_points(pos, cell, grid):
    """Uniform-grid binning of points ``pos`` [dim][n]: (cell of each point, ids sorted by
    (cell, id), cell start, cell one-past-end), empty cells -1."""
    pos = _f64(pos)
    dim, n = pos.shape
    g = _i32(list(grid) + [1] * (3 - len(grid)))
    ncell = int(np.prod(g[:dim]))
    cell_of = np.empty(n, np.int32)
    sid = np.empty(n, np.int32)
    start = np.empty(ncell, np.int32)
    end = np.empty(ncell, np.int32)
    _load().orc_bin_points(dim, n, _ptr(pos), float(cell), _ptr(g), _ptr(cell_of), _ptr(sid), _ptr(start),
                           _ptr(end))
    return cell_of, sid, start, end


def connect(pos, owner, active, npos, radius, cap=None):
    """(owner, neuron) pairs of active cones within ``radius`` of a neuron other than their own.
    ``cap`` sizes the output (default: every pair could connect); a larger count is re-run with
    room for all of it."""
    pos, npos = _f64(pos), _f64(npos)
    dim, n = pos.shape
    m = npos.shape[1]
    owner = _i32(owner)
    act = np.ascontiguousarray(np.ones(n) if active is None else active, dtype=np.uint8)
    cap = n * max(m, 1) if cap is None else int(cap)
    while True:
        src = np.empty(max(cap, 1), np.int32)
        dst = np.empty(max(cap, 1), np.int32)
        k = _load().orc_connect(dim, n, _ptr(pos), _ptr(owner), _ptr(act), m, _ptr(npos), float(radius), cap,
                                _ptr(src), _ptr(dst))
        if k <= cap:
            return src[:k].copy(), dst[:k].copy()
        cap = k


def csr(nv, src, dst):
    """Adjacency list of the distinct edges: (row [nv+1], col [m])."""
    src, dst = _i32(src), _i32(dst)
    row = np.empty(nv + 1, np.int32)
    col = np.empty(max(src.shape[0], 1), np.int32)
    m = _load().orc_csr(nv, src.shape[0], _ptr(src), _ptr(dst), _ptr(row), _ptr(col))
    return row, col[:m].copy()


def bfs(row, col, source):
    """Breadth-first levels from ``source`` (-1 unreachable)."""
    row, col = _i32(row), _i32(col)
    nv = row.shape[0] - 1
    level = np.empty(nv, np.int32)
    _load().orc_bfs(nv, _ptr(row), _ptr(col if col.size else np.zeros(1, np.int32)), int(source), _ptr(level))
    return level
