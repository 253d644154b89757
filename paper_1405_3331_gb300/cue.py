"""Python binding of libcue.so (the C ABI in ``include/cue.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels behind the C ABI.  The functions named like the C entry points take
raw device pointers (ints) and return the C status code; :class:`Simulation`
wraps them around PyTorch-owned device buffers.  There is no CPU fallback:
if the library is missing or fails to load, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np
import threading
from typing import Optional

from . import build as _build

CUE_OK = 0
CUE_ERR_ARG = -1
CUE_ERR_UNSTABLE = -2
CUE_ERR_CUDA = -3
CUE_ERR_NONFINITE = -4
CUE_ERR_TIMEOUT = -5
CUE_ERR_BOUNDS = -6
CUE_ERR_WORKSPACE = -7
CUE_ERR_STATE = -8
CUE_ERR_SCRATCH = -9

CUE_OPT_PATH = 1
CUE_OPT_TEMPORAL_DEPTH = 2
CUE_OPT_ROWS_PER_THREAD = 3
CUE_OPT_TIME_KERNEL = 4
CUE_OPT_PERSIST_ROWS = 5
CUE_OPT_PERSIST_BLOCKS = 6
CUE_OPT_WAIT_LIMIT = 7
CUE_OPT_BARRIER_PHANTOM = 8
CUE_OPT_CLUSTER_CTAS = 9
CUE_INFO_LAST_PATH = 16
CUE_INFO_TILE = 17
CUE_INFO_DEPTH = 18
CUE_INFO_GRID = 19
CUE_INFO_HELPERS = 20
CUE_PATH_AUTO = 0
CUE_PATH_PLAIN = 1
CUE_PATH_FUSED = 2
CUE_PATH_PERSIST = 3
CUE_PATH_RESIDENT = 4
CUE_PATH_CLUSTER = 5

class cue_snr_params(ct.Structure):
    _fields_ = [("gain", ct.c_float), ("width", ct.c_float), ("kd", ct.c_float), ("c_min", ct.c_float),
                ("c_max", ct.c_float), ("turn", ct.c_float)]


EXPORTED = ("cue_set_steering", "cue_workspace_bytes", "cue_init", "cue_step", "cone_step", "sim_run", "cue_get_state",
            "cue_set_state", "cue_set_stream", "cue_set_option", "cue_launch_count", "cue_status",
            "cue_destroy", "cue_strerror", "cue_kernel_time", "cue_cone_updates", "cue_get_option", "sim_run_static",
            "cue_static_scratch_bytes", "cue_static_status", "sim_adjoint", "cue_adjoint_workspace_bytes",
            "cue_adjoint_trace", "cue_endpoint_loss", "cue_set_physics")


class cue_params(ct.Structure):
    _fields_ = [("dim", ct.c_int32), ("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32),
                ("h", ct.c_float), ("D", ct.c_float), ("lam", ct.c_float), ("dt", ct.c_float),
                ("boundary", ct.c_int32)]


class cone_params(ct.Structure):
    _fields_ = [("w_prev", ct.c_float), ("w_grad", ct.c_float), ("w_noise", ct.c_float),
                ("step_len", ct.c_float), ("stop_radius", ct.c_float), ("grad_eps", ct.c_float),
                ("wall_mode", ct.c_int32), ("reserved", ct.c_int32), ("seed", ct.c_uint64)]


class CueError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {cue_strerror(code)} ({code})" if what else
                         f"{cue_strerror(code)} ({code})")


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libcue.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libcue.so not built ({path}); run paper_1405_3331_gb300.build.build()")
            L = ct.CDLL(path)
            P, I32, I64, SZ = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_size_t
            L.cue_workspace_bytes.argtypes = [ct.POINTER(cue_params), I32, I32]
            L.cue_workspace_bytes.restype = SZ
            L.cue_init.argtypes = [ct.POINTER(P), ct.POINTER(cue_params), ct.POINTER(cone_params),
                                   P, P, P, P, I32, P, P, P, P, I32, P, SZ, P]
            for f in ("cue_step", "cone_step", "sim_run"):
                getattr(L, f).argtypes = [P, I32]
            L.cue_get_state.argtypes = [P, ct.POINTER(I64), ct.POINTER(I64), ct.POINTER(I32)]
            L.cue_set_state.argtypes = [P, I64, I64, I32]
            L.cue_set_stream.argtypes = [P, P]
            L.cue_set_option.argtypes = [P, I32, I64]
            L.cue_set_steering.argtypes = [P, ct.POINTER(cue_snr_params)]
            L.cue_set_steering.restype = ct.c_int
            L.cue_get_option.argtypes = [P, I32, ct.POINTER(I64)]
            L.sim_run_static.argtypes = [ct.POINTER(cue_params), ct.POINTER(cone_params), P, P, P, P, I32, P,
                                         P, P, P, I32, I64, I32, P, ct.POINTER(I32)]
            L.sim_run_static.restype = ct.c_int
            L.sim_adjoint.argtypes = [P, P, I32, I32, P, SZ, P, P, P, P, P]
            L.sim_adjoint.restype = ct.c_int
            L.cue_adjoint_workspace_bytes.argtypes = [ct.POINTER(cue_params), I32, I32, I32, I32]
            L.cue_adjoint_workspace_bytes.restype = SZ
            L.cue_adjoint_trace.argtypes = [P, P, P, I64]
            L.cue_adjoint_trace.restype = ct.c_int
            L.cue_endpoint_loss.argtypes = [P, P, P]
            L.cue_endpoint_loss.restype = ct.c_int
            L.cue_set_physics.argtypes = [P, ct.c_float, ct.c_float]
            L.cue_set_physics.restype = ct.c_int
            L.cue_static_scratch_bytes.argtypes = []
            L.cue_static_scratch_bytes.restype = SZ
            L.cue_static_status.argtypes = [P]
            L.cue_static_status.restype = ct.c_int
            L.cue_launch_count.argtypes = [P]
            L.cue_launch_count.restype = ct.c_uint64
            L.cue_status.argtypes = [P]
            L.cue_kernel_time.argtypes = [P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_uint64)]
            L.cue_cone_updates.argtypes = [P, ct.POINTER(ct.c_uint64)]
            L.cue_destroy.argtypes = [P]
            L.cue_destroy.restype = None
            L.cue_strerror.argtypes = [ct.c_int]
            L.cue_strerror.restype = ct.c_char_p
            for f in ("cue_init", "cue_step", "cone_step", "sim_run", "cue_get_state", "cue_set_state",
                      "cue_set_stream", "cue_set_option", "cue_status", "cue_kernel_time",
                      "cue_cone_updates", "cue_get_option"):
                getattr(L, f).restype = ct.c_int
            _lib = L
    return _lib


# ------------------------------------------------------------ C-ABI mirrors
def cue_strerror(code: int) -> str:
    return lib().cue_strerror(int(code)).decode()


def cue_workspace_bytes(params: cue_params, n_src: int, n_axons: int) -> int:
    return int(lib().cue_workspace_bytes(ct.byref(params), n_src, n_axons))


def cue_init(params: cue_params, cone: cone_params, field_a: int, field_b: int, src_cell: int,
             src_emit: int, n_src: int, src_map: int, pos: int, dir: int, active: int, n_axons: int,
             workspace: int, ws_bytes: int, stream: int):
    """Returns (status, handle)."""
    h = ct.c_void_p()
    rc = lib().cue_init(ct.byref(h), ct.byref(params), ct.byref(cone), field_a, field_b, src_cell,
                        src_emit, n_src, src_map or None, pos, dir, active, n_axons, workspace,
                        ws_bytes, stream or None)
    return rc, h


def cue_step(h, nsteps: int) -> int:
    return lib().cue_step(h, nsteps)


def cone_step(h, nsteps: int) -> int:
    return lib().cone_step(h, nsteps)


def sim_run(h, nsteps: int) -> int:
    return lib().sim_run(h, nsteps)


def cue_get_state(h):
    fs, cs, cur = ct.c_int64(), ct.c_int64(), ct.c_int32()
    rc = lib().cue_get_state(h, ct.byref(fs), ct.byref(cs), ct.byref(cur))
    return rc, fs.value, cs.value, cur.value


def cue_set_state(h, field_step: int, cone_step_: int, cur: int) -> int:
    return lib().cue_set_state(h, field_step, cone_step_, cur)


def cue_set_stream(h, stream: int) -> int:
    return lib().cue_set_stream(h, stream or None)


def cue_set_option(h, option: int, value: int) -> int:
    return lib().cue_set_option(h, option, value)


def cue_get_option(h, option: int):
    """Returns (status, value)."""
    v = ct.c_int64()
    rc = lib().cue_get_option(h, option, ct.byref(v))
    return rc, v.value


def cue_launch_count(h) -> int:
    return int(lib().cue_launch_count(h))


def cue_status(h) -> int:
    return lib().cue_status(h)


def cue_kernel_time(h):
    """Returns (status, total_ms, launches) of the dominant kernel since the last call."""
    ms, n = ct.c_double(), ct.c_uint64()
    rc = lib().cue_kernel_time(h, ct.byref(ms), ct.byref(n))
    return rc, ms.value, n.value


def cue_cone_updates(h):
    """Returns (status, count) of cone updates since the last call."""
    n = ct.c_uint64()
    rc = lib().cue_cone_updates(h, ct.byref(n))
    return rc, n.value


def sim_run_static(params: cue_params, cone: cone_params, field_a: int, field_b: int, src_cell: int,
                   src_emit: int, n_src: int, src_map: int, pos: int, dir: int, active: int, n_axons: int,
                   step0: int, nsteps: int, stream: int):
    """The coupled run without a caller workspace (fixed device scratch array).

    Returns (status, index of the buffer holding the result)."""
    cur = ct.c_int32(-1)
    rc = lib().sim_run_static(ct.byref(params), ct.byref(cone), field_a, field_b, src_cell, src_emit, n_src,
                              src_map or None, pos, dir, active, n_axons, step0, nsteps, stream or None,
                              ct.byref(cur))
    return rc, cur.value


def cue_adjoint_workspace_bytes(params: cue_params, n_src: int, n_axons: int, nsteps: int,
                                ckpt_every: int) -> int:
    return int(lib().cue_adjoint_workspace_bytes(ct.byref(params), n_src, n_axons, nsteps, ckpt_every))


def sim_adjoint(h, targets: int, nsteps: int, ckpt_every: int, ws: int, ws_bytes: int, gD: int, glam: int,
                gsrc: int, gmap: int, loss: int) -> int:
    return lib().sim_adjoint(h, targets, nsteps, ckpt_every, ws, ws_bytes, gD, glam, gsrc or None,
                             gmap or None, loss)


def cue_endpoint_loss(h, targets: int, loss: int) -> int:
    return lib().cue_endpoint_loss(h, targets or None, loss)


def cue_set_physics(h, D: float, lam: float) -> int:
    return lib().cue_set_physics(h, D, lam)


def cue_adjoint_trace(h, fields: int, cones: int, max_states: int) -> int:
    return lib().cue_adjoint_trace(h, fields or None, cones or None, max_states)


def cue_static_scratch_bytes() -> int:
    return int(lib().cue_static_scratch_bytes())


def cue_static_status(stream: int) -> int:
    """Synchronise ``stream``, then return and clear the status word of sim_run_static's scratch."""
    return lib().cue_static_status(stream or None)


def cue_destroy(h) -> None:
    lib().cue_destroy(h)


def _check(rc: int, what: str):
    if rc != CUE_OK:
        raise CueError(rc, what)


# ------------------------------------------------------------ tensor wrapper
class Simulation:
    """A simulation over PyTorch-owned device buffers.

    ``workload`` is a :class:`paper_1405_3331_gb300.workloads.Workload` (or
    anything with the same attributes).  All buffers live on ``device``; the
    library runs on ``stream`` (default: the current torch stream).  ``field_offset``
    places the two field buffers that many floats into their allocations; an offset
    that is not a multiple of 4 breaks 16-byte alignment and so selects the any-size
    kernels (used by the tests to compare kernels bit for bit).
    """

    def __init__(self, workload, device="cuda:0", stream=None, path: int = CUE_PATH_AUTO,
                 field_offset: int = 0):
        import torch
        self.torch = torch
        self.w = workload
        self.device = torch.device(device)
        wl = workload
        self.dim = wl.dim
        shape = wl.shape
        self.params = cue_params(wl.dim, wl.nx, wl.ny, wl.nz if wl.dim == 3 else 1, wl.h, wl.D,
                                 wl.lam, wl.dt, 0)
        self.cone = cone_params(wl.w_prev, wl.w_grad, wl.w_noise, wl.step_len, wl.stop_radius,
                                wl.grad_eps, wl.wall_mode, 0, wl.seed & 0xFFFFFFFFFFFFFFFF)
        dev = self.device
        with torch.cuda.device(dev):
            n_cells = int(np.prod(shape))
            self._field_store = [torch.empty(n_cells + field_offset, dtype=torch.float32, device=dev)
                                 for _ in range(2)]
            self.fields = [st[field_offset:].view(shape) for st in self._field_store]
            self.fields[0].copy_(torch.as_tensor(wl.field0()))
            self.src_cell = torch.as_tensor(wl.src_cell, dtype=torch.int32, device=dev)
            self.src_emit = torch.as_tensor(wl.src_emit, dtype=torch.float32, device=dev)
            self.src_map = (None if wl.src_map is None else
                            torch.as_tensor(wl.src_map, dtype=torch.float32, device=dev).contiguous())
            self.pos = torch.as_tensor(wl.pos, dtype=torch.float32, device=dev).contiguous()
            self.dir = torch.as_tensor(wl.dir, dtype=torch.float32, device=dev).contiguous()
            self.active = torch.as_tensor(wl.active, dtype=torch.uint8, device=dev).contiguous()
            self.n_src = int(self.src_cell.numel())
            self.n_axons = int(self.active.numel())
            self.ws_bytes = cue_workspace_bytes(self.params, self.n_src, self.n_axons)
            if self.ws_bytes == 0:
                raise CueError(CUE_ERR_ARG, "cue_workspace_bytes")
            self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=dev)
            ws_ptr = (self.workspace.data_ptr() + 255) & ~255
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            rc, self.h = cue_init(self.params, self.cone, self.fields[0].data_ptr(),
                                  self.fields[1].data_ptr(), self.src_cell.data_ptr(),
                                  self.src_emit.data_ptr(), self.n_src,
                                  0 if self.src_map is None else self.src_map.data_ptr(),
                                  self.pos.data_ptr(), self.dir.data_ptr(), self.active.data_ptr(),
                                  self.n_axons, ws_ptr, self.ws_bytes, self.stream.cuda_stream)
            _check(rc, "cue_init")
        if path != CUE_PATH_AUTO:
            self.set_option(CUE_OPT_PATH, path)

    # -- stepping
    def sim_run(self, nsteps: int):
        _check(sim_run(self.h, nsteps), "sim_run")

    def cue_step(self, nsteps: int):
        _check(cue_step(self.h, nsteps), "cue_step")

    def cone_step(self, nsteps: int):
        _check(cone_step(self.h, nsteps), "cone_step")

    def status(self) -> int:
        return cue_status(self.h)

    def check(self):
        _check(self.status(), "cue_status")

    def set_option(self, option: int, value: int):
        _check(cue_set_option(self.h, option, value), "cue_set_option")

    def set_steering(self, snr=None):
        """None: vector-addition steering; else a dict / object with gain, width, kd, c_min,
        c_max, turn for the SNR turn rule (2D)."""
        if snr is None:
            _check(lib().cue_set_steering(self.h, None), "cue_set_steering")
            return
        get = (lambda k: snr[k]) if isinstance(snr, dict) else (lambda k: getattr(snr, k))
        p = cue_snr_params(get("gain"), get("width"), get("kd"), get("c_min"), get("c_max"), get("turn"))
        _check(lib().cue_set_steering(self.h, ct.byref(p)), "cue_set_steering")

    def get_option(self, option: int) -> int:
        rc, v = cue_get_option(self.h, option)
        _check(rc, "cue_get_option")
        return v

    def fused_active(self) -> bool:
        """True when the last stepping call ran on the fused, temporally blocked path."""
        return self.get_option(CUE_INFO_LAST_PATH) == CUE_PATH_FUSED

    def last_path(self) -> int:
        """CUE_PATH_PLAIN, CUE_PATH_FUSED, CUE_PATH_PERSIST, CUE_PATH_RESIDENT or CUE_PATH_CLUSTER:
        the path of the last sim_run."""
        return self.get_option(CUE_INFO_LAST_PATH)

    def launches(self) -> int:
        return cue_launch_count(self.h)

    def cone_updates(self) -> int:
        """Active cone x step updates since the last call (synchronises)."""
        rc, n = cue_cone_updates(self.h)
        _check(rc, "cue_cone_updates")
        return n

    def kernel_time(self):
        """(total_ms, launches) of the dominant kernel since the last call (needs
        CUE_OPT_TIME_KERNEL)."""
        rc, ms, n = cue_kernel_time(self.h)
        _check(rc, "cue_kernel_time")
        return ms, n

    # -- state
    def state(self):
        rc, fs, cs, cur = cue_get_state(self.h)
        _check(rc, "cue_get_state")
        return fs, cs, cur

    def field(self):
        """The tensor holding the current field (a view of the library's buffer)."""
        return self.fields[self.state()[2]]

    def load(self, C=None, pos=None, dir=None, active=None, step: Optional[int] = None):
        """Overwrite the state (host arrays or tensors) and, optionally, both step counters."""
        torch = self.torch
        fs, cs, cur = self.state()
        if C is not None:
            self.fields[cur].copy_(torch.as_tensor(C, dtype=torch.float32).reshape(self.fields[cur].shape))
        if pos is not None:
            self.pos.copy_(torch.as_tensor(pos, dtype=torch.float32))
        if dir is not None:
            self.dir.copy_(torch.as_tensor(dir, dtype=torch.float32))
        if active is not None:
            self.active.copy_(torch.as_tensor(active, dtype=torch.uint8))
        if step is not None:
            _check(cue_set_state(self.h, step, step, cur), "cue_set_state")
        torch.cuda.synchronize(self.device)

    def snapshot(self):
        """(C, pos, dir, active, field_step, cone_step) as numpy arrays (synchronises)."""
        self.torch.cuda.synchronize(self.device)
        fs, cs, cur = self.state()
        return (self.fields[cur].cpu().numpy(), self.pos.cpu().numpy(), self.dir.cpu().numpy(),
                self.active.cpu().numpy(), fs, cs)

    def adjoint(self, targets, nsteps: int, ckpt_every: int = 64, want_map: bool = True, trace: bool = False):
        """Gradients of L = mean_a |p_a(T) - t_a|^2 after ``nsteps`` more steps (no-stopping
        runs only).  Returns a dict of device tensors: loss, dD, dlambda, dsrc, dmap (or None);
        with ``trace`` also ``trace_C`` (nsteps + 1, *shape) and ``trace_cone`` (nsteps + 1, 2,
        dim, n_axons): the FP32 forward states the backward pass read (cue_adjoint_trace).
        The handle advances by ``nsteps``, as with sim_run."""
        torch = self.torch
        dev = self.device
        tg = torch.as_tensor(targets, dtype=torch.float32, device=dev).contiguous()
        tr = None
        if trace:
            tr = (torch.empty((nsteps + 1,) + tuple(self.fields[0].shape), dtype=torch.float32, device=dev),
                  torch.empty((nsteps + 1, 2, self.dim, self.n_axons), dtype=torch.float32, device=dev))
            _check(cue_adjoint_trace(self.h, tr[0].data_ptr(), tr[1].data_ptr(), nsteps + 1), "cue_adjoint_trace")
        nbytes = cue_adjoint_workspace_bytes(self.params, self.n_src, self.n_axons, nsteps, ckpt_every)
        if nbytes == 0:
            raise CueError(CUE_ERR_ARG, "cue_adjoint_workspace_bytes")
        ws = getattr(self, "_adj_ws", None)           # one adjoint workspace, reused while it is big enough
        if ws is None or ws.numel() < nbytes + 256:
            ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            self._adj_ws = ws
        ws_ptr = (ws.data_ptr() + 255) & ~255
        out = {k: torch.zeros((), dtype=torch.float32, device=dev) for k in ("loss", "dD", "dlambda")}
        out["dsrc"] = torch.zeros(max(self.n_src, 1), dtype=torch.float32, device=dev)
        out["dmap"] = torch.zeros(self.fields[0].shape, dtype=torch.float32, device=dev) if want_map else None
        rc = sim_adjoint(self.h, tg.data_ptr(), nsteps, ckpt_every, ws_ptr, nbytes, out["dD"].data_ptr(),
                         out["dlambda"].data_ptr(), out["dsrc"].data_ptr() if self.n_src else 0,
                         out["dmap"].data_ptr() if want_map else 0, out["loss"].data_ptr())
        if trace:
            _check(cue_adjoint_trace(self.h, 0, 0, 0), "cue_adjoint_trace")
        _check(rc, "sim_adjoint")
        self._adj_keep = (ws, tg)            # keep the buffers alive until the stream has used them
        out["dsrc"] = out["dsrc"][: self.n_src]
        if trace:
            out["trace_C"], out["trace_cone"] = tr
        return out

    def run_host(self, C, pos, dir, active, nsteps: int, out=None):
        """End-to-end call from host memory: copy the state in (pinned host tensors copy
        asynchronously), advance ``nsteps`` coupled steps, copy the state back into ``out``
        (C, pos, dir, active host tensors, allocated pinned when None).  Both step counters
        restart at 0.  Returns ``out`` after synchronising the stream."""
        torch = self.torch
        with torch.cuda.stream(self.stream):
            self.fields[0].copy_(torch.as_tensor(C).reshape(self.fields[0].shape), non_blocking=True)
            self.pos.copy_(torch.as_tensor(pos), non_blocking=True)
            self.dir.copy_(torch.as_tensor(dir), non_blocking=True)
            self.active.copy_(torch.as_tensor(active), non_blocking=True)
            _check(cue_set_state(self.h, 0, 0, 0), "cue_set_state")
            self.sim_run(nsteps)
            cur = self.state()[2]
            if out is None:
                out = tuple(torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                            for t in (self.fields[0], self.pos, self.dir, self.active))
            out[0].copy_(self.fields[cur], non_blocking=True)
            out[1].copy_(self.pos, non_blocking=True)
            out[2].copy_(self.dir, non_blocking=True)
            out[3].copy_(self.active, non_blocking=True)
        self.stream.synchronize()
        return out

    def close(self):
        if getattr(self, "h", None):
            cue_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
