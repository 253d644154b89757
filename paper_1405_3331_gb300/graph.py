"""Python binding of include/cue_graph.h: uniform-grid binning, growth-cone / neuron
connections, the adjacency list and breadth-first levels (argument marshalling over
PyTorch-owned device buffers; every step runs in libcue.so)."""
from __future__ import annotations

import ctypes as ct

from . import cue as _cue
from .cue import CueError

EXPORTED = ("cue_bin_workspace_bytes", "cue_bin_points", "cue_connect", "cue_csr_workspace_bytes",
            "cue_csr_build", "cue_bfs_workspace_bytes", "cue_bfs", "cue_graph_status")

_declared = False


def _lib():
    global _declared
    L = _cue.lib()
    if not _declared:
        P, I32, I64, F, SZ = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_float, ct.c_size_t
        L.cue_bin_workspace_bytes.argtypes = [I32, I64]
        L.cue_bin_workspace_bytes.restype = SZ
        L.cue_bin_points.argtypes = [I32, I32, P, F, P, P, P, P, P, P, SZ, P]
        L.cue_connect.argtypes = [I32, I32, P, P, P, I32, P, F, F, P, P, P, P, I32, P, P, P, P]
        L.cue_csr_workspace_bytes.argtypes = [I32, I32]
        L.cue_csr_workspace_bytes.restype = SZ
        L.cue_csr_build.argtypes = [I32, I32, P, P, P, P, P, P, P, SZ, P]
        L.cue_bfs_workspace_bytes.argtypes = [I32]
        L.cue_bfs_workspace_bytes.restype = SZ
        L.cue_bfs.argtypes = [I32, P, P, I32, P, P, SZ, P]
        L.cue_graph_status.argtypes = [P, P]
        for f in ("cue_bin_points", "cue_connect", "cue_csr_build", "cue_bfs", "cue_graph_status"):
            getattr(L, f).restype = ct.c_int
        _declared = True
    return L


def _check(rc, what):
    if rc != _cue.CUE_OK:
        raise CueError(rc, what)


def _ws(torch, nbytes, device):
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    return buf, (buf.data_ptr() + 255) & ~255


def _grid(grid):
    return (ct.c_int32 * 3)(*(list(grid) + [1] * (3 - len(grid))))


def bin_points(pos, cell: float, grid, stream=None):
    """pos: float32 device tensor [dim, n].  Returns (cell_of, sorted_id, cell_start, cell_end)."""
    import torch
    dim, n = pos.shape
    ncell = 1
    for g in grid[:dim]:
        ncell *= int(g)
    dev = pos.device
    out = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(2)]
    out += [torch.empty(ncell, dtype=torch.int32, device=dev) for _ in range(2)]
    L = _lib()
    nbytes = int(L.cue_bin_workspace_bytes(n, ncell))
    buf, ws = _ws(torch, nbytes, dev)
    st = (stream or torch.cuda.current_stream(dev)).cuda_stream
    _check(L.cue_bin_points(dim, n, pos.data_ptr(), float(cell), _grid(grid), *[t.data_ptr() for t in out], ws,
                            nbytes, st), "cue_bin_points")
    torch.cuda.synchronize(dev)                      # the workspace is released on return
    del buf
    return tuple(out)


def connect(pos, owner, active, npos, radius: float, cell: float, grid, binned, cap: int, stream=None):
    """Connections of cones ``pos`` [dim, n] to neurons ``npos`` binned by :func:`bin_points`.
    Returns (src, dst, count) device tensors (count is a 1-element tensor)."""
    import torch
    dim, n = pos.shape
    m = npos.shape[1]
    dev = pos.device
    src = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    dst = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    _, sid, start, end = binned
    st = (stream or torch.cuda.current_stream(dev)).cuda_stream
    _check(_lib().cue_connect(dim, n, pos.data_ptr(), owner.data_ptr(), active.data_ptr() if active is not None else None,
                              m, npos.data_ptr(), float(radius), float(cell), _grid(grid), sid.data_ptr(),
                              start.data_ptr(), end.data_ptr(), cap, src.data_ptr(), dst.data_ptr(), cnt.data_ptr(), st),
           "cue_connect")
    return src, dst, cnt


def csr(nv: int, src, dst, count, stream=None):
    """Adjacency list of the distinct edges among the first ``count`` (device tensor) pairs.
    Returns (row [nv+1], col [cap], m) device tensors."""
    import torch
    dev = src.device
    cap = src.shape[0]
    row = torch.empty(nv + 1, dtype=torch.int32, device=dev)
    col = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    m = torch.zeros(1, dtype=torch.int32, device=dev)
    L = _lib()
    nbytes = int(L.cue_csr_workspace_bytes(nv, cap))
    buf, ws = _ws(torch, nbytes, dev)
    st = (stream or torch.cuda.current_stream(dev)).cuda_stream
    _check(L.cue_csr_build(nv, cap, count.data_ptr(), src.data_ptr(), dst.data_ptr(), row.data_ptr(), col.data_ptr(),
                           m.data_ptr(), ws, nbytes, st), "cue_csr_build")
    torch.cuda.synchronize(dev)
    del buf
    return row, col, m


def bfs(row, col, source: int, stream=None):
    """Breadth-first levels from ``source`` (-1 unreachable) as an int32 device tensor."""
    import torch
    dev = row.device
    nv = row.shape[0] - 1
    level = torch.empty(max(nv, 1), dtype=torch.int32, device=dev)
    L = _lib()
    nbytes = int(L.cue_bfs_workspace_bytes(nv))
    buf, ws = _ws(torch, nbytes, dev)
    st = (stream or torch.cuda.current_stream(dev)).cuda_stream
    _check(L.cue_bfs(nv, row.data_ptr(), col.data_ptr(), int(source), level.data_ptr(), ws, nbytes, st), "cue_bfs")
    _check(L.cue_graph_status(ws, st), "cue_graph_status")
    del buf
    return level[:nv]
