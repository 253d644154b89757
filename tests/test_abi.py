"""libcue.so builds, loads, exports every entry point of include/cue.h, and its
host-side argument checks answer without touching a GPU."""
import ctypes as ct
import os
import re
import subprocess

import pytest

from paper_1405_3331_gb300 import build as cue_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def cue():
    cue_build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\**\s*([A-Za-z_]\w*)\s*\(",
                             text, flags=re.M):
            if m.group(1) not in ("if", "defined"):
                names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("cue_init", "cue_step", "cone_step", "sim_run", "cue_status", "cue_destroy",
                 "cue_strerror", "cue_workspace_bytes"):
        assert must in names


def test_library_exports_every_declared_symbol(cue):
    out = subprocess.run(["nm", "-D", "--defined-only", cue.lib_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = cue.lib()
    for n in declared_functions():
        assert hasattr(L, n)
    assert set(cue.EXPORTED) <= set(declared_functions())


def test_binding_constants_match_the_headers(cue):
    """Every CUE_* constant of the Python binding has its header's value (paths, options,
    error codes)."""
    defines = {}
    for h in HEADERS:
        for m in re.finditer(r"^#define\s+(CUE_\w+)\s+\(?(-?\d+)\)?", open(h).read(), flags=re.M):
            defines[m.group(1)] = int(m.group(2))
    consts = {k: v for k, v in vars(cue).items() if k.startswith("CUE_") and isinstance(v, int)}
    assert "CUE_PATH_RESIDENT" in consts and "CUE_PATH_RESIDENT" in defines
    mismatched = {k: (v, defines[k]) for k, v in consts.items() if k in defines and defines[k] != v}
    assert not mismatched, mismatched
    assert len(set(consts) & set(defines)) >= 20


def test_strerror_covers_every_code(cue):
    for code in range(0, -10, -1):
        s = cue.cue_strerror(code)
        assert s and s != "unknown status code"
    assert cue.cue_strerror(-99) == "unknown status code"


def _params(cue, **kw):
    d = dict(dim=2, nx=64, ny=48, nz=1, h=1.0, D=1.0, lam=0.01, dt=0.2, boundary=0)
    d.update(kw)
    return cue.cue_params(d["dim"], d["nx"], d["ny"], d["nz"], d["h"], d["D"], d["lam"], d["dt"],
                          d["boundary"])


def _cone(cue, **kw):
    d = dict(w_prev=0.5, w_grad=0.4, w_noise=0.1, step_len=0.5, stop_radius=0.0, grad_eps=1e-15,
             wall_mode=0, reserved=0, seed=7)
    d.update(kw)
    return cue.cone_params(*d.values())


def test_workspace_bytes(cue):
    ws = cue.cue_workspace_bytes(_params(cue), 4, 64)
    assert ws > 0 and ws % 256 == 0
    assert cue.cue_workspace_bytes(_params(cue), 400, 64000) > ws
    assert cue.cue_workspace_bytes(_params(cue, dim=4), 4, 64) == 0
    assert cue.cue_workspace_bytes(_params(cue, nx=1), 4, 64) == 0
    assert cue.cue_workspace_bytes(_params(cue), -1, 64) == 0


FAKE = 0x10000      # never dereferenced: every case below fails validation first


def _init(cue, params, cone, fa=FAKE, fb=FAKE * 2, n_src=1, n_ax=1, ws=FAKE * 4, ws_bytes=1 << 20,
          map_=0, ptr=FAKE * 8):
    return cue.cue_init(params, cone, fa, fb, ptr, ptr, n_src, map_, ptr, ptr, ptr, n_ax, ws, ws_bytes, 0)[0]


@pytest.mark.parametrize("bad", [
    dict(dim=1), dict(dim=4), dict(nx=1), dict(ny=0), dict(dim=3, nz=1), dict(h=0.0), dict(h=-1.0),
    dict(dt=0.0), dict(D=-1.0), dict(lam=-0.1), dict(boundary=1), dict(h=float("nan")),
])
def test_init_rejects_bad_params(cue, bad):
    assert _init(cue, _params(cue, **bad), _cone(cue)) == cue.CUE_ERR_ARG


@pytest.mark.parametrize("bad", [dict(wall_mode=2), dict(reserved=1), dict(step_len=-1.0),
                                 dict(grad_eps=-1.0), dict(w_grad=float("inf"))])
def test_init_rejects_bad_cone(cue, bad):
    assert _init(cue, _params(cue), _cone(cue, **bad)) == cue.CUE_ERR_ARG


def test_init_rejects_bad_pointers(cue):
    p, c = _params(cue), _cone(cue)
    assert _init(cue, p, c, fa=0) == cue.CUE_ERR_ARG
    assert _init(cue, p, c, fa=FAKE, fb=FAKE) == cue.CUE_ERR_ARG
    assert _init(cue, p, c, ptr=0) == cue.CUE_ERR_ARG
    assert _init(cue, p, c, n_src=-1) == cue.CUE_ERR_ARG
    # null out-pointer
    assert cue.lib().cue_init(None, ct.byref(p), ct.byref(c), FAKE, FAKE * 2, FAKE, FAKE, 1, None, FAKE,
                              FAKE, FAKE, 1, FAKE, 1 << 20, None) == cue.CUE_ERR_ARG


@pytest.mark.parametrize("dim,D,dt,h,lam", [(2, 1.0, 0.26, 1.0, 0.0), (3, 1.0, 0.17, 1.0, 0.0),
                                             (2, 1.0, 0.2, 0.5, 0.0), (2, 0.0, 0.2, 1.0, 6.0)])
def test_init_rejects_unstable(cue, dim, D, dt, h, lam):
    p = _params(cue, dim=dim, nz=8, D=D, dt=dt, h=h, lam=lam)
    assert _init(cue, p, _cone(cue)) == cue.CUE_ERR_UNSTABLE


def test_init_rejects_small_or_misaligned_workspace(cue):
    p, c = _params(cue), _cone(cue)
    need = cue.cue_workspace_bytes(p, 1, 1)
    assert _init(cue, p, c, ws_bytes=need - 1) == cue.CUE_ERR_WORKSPACE
    assert _init(cue, p, c, ws=FAKE * 4 + 16, ws_bytes=need) == cue.CUE_ERR_WORKSPACE
    assert _init(cue, p, c, ws=0, ws_bytes=need) == cue.CUE_ERR_WORKSPACE


def test_calls_on_null_handle(cue):
    L = cue.lib()
    assert L.sim_run(None, 1) == cue.CUE_ERR_ARG
    assert L.cue_step(None, 1) == cue.CUE_ERR_ARG
    assert L.cone_step(None, 1) == cue.CUE_ERR_ARG
    assert L.cue_status(None) == cue.CUE_ERR_ARG
    assert L.cue_set_option(None, 1, 0) == cue.CUE_ERR_ARG
    assert L.cue_launch_count(None) == 0
    L.cue_destroy(None)


def test_batch_host_checks_answer_without_a_gpu(cue):
    from paper_1405_3331_gb300 import batch
    L = batch._lib()
    inst = (batch.cue_instance * 2)()
    for I in inst:
        I.params = _params(cue, nx=66, ny=40)
        I.cone = _cone(cue)
        I.pitch = 68
        I.field_a, I.field_b = 0x100000, 0x200000         # never dereferenced by the host checks
        I.pos, I.dir, I.active = 0x300000, 0x400000, 0x500000
        I.n_axons = 10
    ws = L.cue_batch_workspace_bytes(2, inst, 0)
    ws_bk = L.cue_batch_workspace_bytes(2, inst, 1)
    assert ws > 0 and ws % 256 == 0 and ws_bk > ws
    inst[1].pitch = 64                                     # pitch < nx
    assert L.cue_batch_workspace_bytes(2, inst, 0) == 0
    err = ct.c_int32(0)
    assert not L.cue_batch_create(2, inst, None, 0, None, ct.byref(err))
    assert err.value == cue.CUE_ERR_ARG
    inst[1].pitch = 66                                     # not a multiple of 4
    assert not L.cue_batch_create(2, inst, None, 0, None, ct.byref(err))
    assert err.value == cue.CUE_ERR_ARG
    inst[1].pitch = 68
    inst[1].params = _params(cue, nx=66, ny=40, D=5.0)    # alpha = 1 > 1/4
    assert not L.cue_batch_create(2, inst, None, 0, None, ct.byref(err))
    assert err.value == cue.CUE_ERR_UNSTABLE
    inst[1].params = _params(cue, nx=66, ny=40)
    assert not L.cue_batch_create(2, inst, None, 0, None, ct.byref(err))   # no workspace
    assert err.value == cue.CUE_ERR_WORKSPACE
    assert L.cue_batch_run(None, 1) == cue.CUE_ERR_ARG
