"""Python binding of include/cue_batch.h: many independent 2D simulations of
uneven sizes stepped together -- one persistent launch, one launch per step, or
temporally blocked launches (argument marshalling over PyTorch-owned device
buffers; every step runs in libcue.so)."""
from __future__ import annotations

import ctypes as ct
from typing import List, Sequence

import numpy as np

from . import cue as _cue
from .cue import CueError, cone_params, cue_params

CUE_BOPT_ROWS = 1
CUE_BOPT_BLOCKS = 2
CUE_BOPT_GRAPH = 3
CUE_BOPT_MODE = 4
CUE_BOPT_DEPTH = 5
CUE_BINFO_ITEMS = 16
CUE_BINFO_STEP = 17
CUE_BINFO_CUR = 18
CUE_BINFO_GRID = 19
CUE_BINFO_BLOCKED = 20

EXPORTED = ("cue_batch_workspace_bytes", "cue_batch_create", "cue_batch_run", "cue_batch_autotune",
            "cue_batch_set_state", "cue_batch_set_option", "cue_batch_get_option", "cue_batch_status",
            "cue_batch_cone_updates", "cue_batch_destroy")


class cue_instance(ct.Structure):
    _fields_ = [("params", cue_params), ("cone", cone_params), ("pitch", ct.c_int32),
                ("field_a", ct.c_void_p), ("field_b", ct.c_void_p), ("src_cell", ct.c_void_p),
                ("src_emit", ct.c_void_p), ("n_src", ct.c_int32), ("src_map", ct.c_void_p),
                ("pos", ct.c_void_p), ("dir", ct.c_void_p), ("active", ct.c_void_p), ("n_axons", ct.c_int32)]


_declared = False


def _lib():
    global _declared
    L = _cue.lib()
    if not _declared:
        P, I32, I64 = ct.c_void_p, ct.c_int32, ct.c_int64
        L.cue_batch_workspace_bytes.argtypes = [I32, ct.POINTER(cue_instance), I32]
        L.cue_batch_workspace_bytes.restype = ct.c_size_t
        L.cue_batch_create.argtypes = [I32, ct.POINTER(cue_instance), P, ct.c_size_t, P, ct.POINTER(I32)]
        L.cue_batch_create.restype = P
        L.cue_batch_run.argtypes = [P, I32]
        L.cue_batch_autotune.argtypes = [P, I32, ct.POINTER(I32), ct.POINTER(I32), ct.POINTER(ct.c_double)]
        L.cue_batch_set_option.argtypes = [P, I32, I64]
        L.cue_batch_set_state.argtypes = [P, I64, I32]
        L.cue_batch_get_option.argtypes = [P, I32, ct.POINTER(I64)]
        L.cue_batch_status.argtypes = [P]
        L.cue_batch_cone_updates.argtypes = [P, ct.POINTER(ct.c_uint64)]
        L.cue_batch_destroy.argtypes = [P]
        L.cue_batch_destroy.restype = None
        for f in ("cue_batch_run", "cue_batch_autotune", "cue_batch_set_state", "cue_batch_set_option",
                  "cue_batch_get_option",
                  "cue_batch_status", "cue_batch_cone_updates"):
            getattr(L, f).restype = ct.c_int
        _declared = True
    return L


def _check(rc: int, what: str):
    if rc != _cue.CUE_OK:
        raise CueError(rc, what)


class Batch:
    """Workloads (2D, see :mod:`paper_1405_3331_gb300.workloads`) as one batch on ``device``.
    Fields are stored with a row pitch rounded up to a multiple of 4."""

    def __init__(self, workloads: Sequence, device="cuda:0", stream=None, backup: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.w = list(workloads)
        self._keep = []
        inst = (cue_instance * len(self.w))()
        self.fields, self.pos, self.dir, self.active, self.pitch = [], [], [], [], []
        with torch.cuda.stream(self.stream):
            for i, w in enumerate(self.w):
                if w.dim != 2:
                    raise ValueError("batched runs are 2D")
                pitch = (w.nx + 3) // 4 * 4
                fa = torch.zeros((w.ny, pitch), dtype=torch.float32, device=self.device)
                fa[:, : w.nx] = torch.as_tensor(w.field0(), device=self.device)
                fb = torch.zeros_like(fa)
                cell = torch.as_tensor(w.src_cell, dtype=torch.int32, device=self.device)
                emit = torch.as_tensor(w.src_emit, dtype=torch.float32, device=self.device)
                smap = None
                if w.src_map is not None:
                    smap = torch.zeros((w.ny, pitch), dtype=torch.float32, device=self.device)
                    smap[:, : w.nx] = torch.as_tensor(w.src_map, device=self.device)
                pos = torch.as_tensor(w.pos, dtype=torch.float32, device=self.device).contiguous()
                dirs = torch.as_tensor(w.dir, dtype=torch.float32, device=self.device).contiguous()
                act = torch.as_tensor(w.active, dtype=torch.uint8, device=self.device).contiguous()
                self._keep += [fa, fb, cell, emit, smap, pos, dirs, act]
                self.fields.append((fa, fb))
                self.pos.append(pos)
                self.dir.append(dirs)
                self.active.append(act)
                self.pitch.append(pitch)
                I = inst[i]
                I.params = cue_params(2, w.nx, w.ny, 1, w.h, w.D, w.lam, w.dt, 0)
                I.cone = cone_params(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps,
                                     w.wall_mode, 0, w.seed)
                I.pitch = pitch
                I.field_a, I.field_b = fa.data_ptr(), fb.data_ptr()
                I.src_cell = cell.data_ptr() if w.n_src else None
                I.src_emit = emit.data_ptr() if w.n_src else None
                I.n_src = w.n_src
                I.src_map = smap.data_ptr() if smap is not None else None
                I.pos, I.dir, I.active = pos.data_ptr(), dirs.data_ptr(), act.data_ptr()
                I.n_axons = w.n_axons
        self.stream.synchronize()
        L = _lib()
        nbytes = int(L.cue_batch_workspace_bytes(len(self.w), inst, 1 if backup else 0))
        if nbytes == 0:
            raise CueError(_cue.CUE_ERR_ARG, "cue_batch_workspace_bytes")
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ws_ptr = (self.ws.data_ptr() + 255) & ~255
        err = ct.c_int32(0)
        h = L.cue_batch_create(len(self.w), inst, ws_ptr, nbytes, self.stream.cuda_stream, ct.byref(err))
        if not h:
            raise CueError(err.value, "cue_batch_create")
        self.h = ct.c_void_p(h)
        self._inst = inst

    # -- calls
    def run(self, nsteps: int):
        _check(_lib().cue_batch_run(self.h, nsteps), "cue_batch_run")

    def autotune(self, probe_steps: int = 20):
        r, b, ms = ct.c_int32(), ct.c_int32(), ct.c_double()
        _check(_lib().cue_batch_autotune(self.h, probe_steps, ct.byref(r), ct.byref(b), ct.byref(ms)),
               "cue_batch_autotune")
        return r.value, b.value, ms.value

    def set_option(self, option: int, value: int):
        _check(_lib().cue_batch_set_option(self.h, option, value), "cue_batch_set_option")

    def reset_state(self, step: int = 0, cur: int = 0):
        """Every instance back to step ``step`` with buffer ``cur`` (0 = the first) current."""
        _check(_lib().cue_batch_set_state(self.h, step, cur), "cue_batch_set_state")

    def get_option(self, option: int) -> int:
        v = ct.c_int64()
        _check(_lib().cue_batch_get_option(self.h, option, ct.byref(v)), "cue_batch_get_option")
        return v.value

    def status(self) -> int:
        return _lib().cue_batch_status(self.h)

    def check(self):
        _check(self.status(), "cue_batch_status")

    def cone_updates(self) -> int:
        n = ct.c_uint64()
        _check(_lib().cue_batch_cone_updates(self.h, ct.byref(n)), "cue_batch_cone_updates")
        return n.value

    def snapshot(self, i: int):
        """Instance i: (C [ny, nx], pos, dir, active) as numpy arrays (synchronises)."""
        self.stream.synchronize()
        cur = self.get_option(CUE_BINFO_CUR)
        w = self.w[i]
        C = self.fields[i][cur][:, : w.nx].cpu().numpy()
        return C, self.pos[i].cpu().numpy(), self.dir[i].cpu().numpy(), self.active[i].cpu().numpy()

    def n_cells(self) -> int:
        return int(sum(w.n_cells for w in self.w))

    def close(self):
        if getattr(self, "h", None):
            _lib().cue_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
