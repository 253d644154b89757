"""sim_run_static: the coupled run for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (code running under another framework's
allocator, hosts that forbid device allocation after start-up); this entry
point takes no workspace and keeps its scratch in a fixed device array inside
the library.  Its results must equal sim_run's bit for bit on the same state,
over two calls in a row (the second continues where the first stopped, on the
scratch the first call left behind), and device-side problems must come back
through cue_static_status.  The file name keeps it last in collection.
"""
import numpy as np
import pytest

from paper_1405_3331_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cue():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


def _buffers(torch, w):
    dev = torch.device("cuda:0")
    return dict(
        fields=[torch.as_tensor(w.field0(), device=dev).contiguous(),
                torch.zeros(w.shape, dtype=torch.float32, device=dev)],
        src_cell=torch.as_tensor(w.src_cell, dtype=torch.int32, device=dev),
        src_emit=torch.as_tensor(w.src_emit, dtype=torch.float32, device=dev),
        src_map=None if w.src_map is None else torch.as_tensor(w.src_map, device=dev).contiguous(),
        pos=torch.as_tensor(w.pos, device=dev).contiguous(),
        dir=torch.as_tensor(w.dir, device=dev).contiguous(),
        active=torch.as_tensor(w.active, device=dev).contiguous())


def _static_call(cue, torch, sim, b, step0, nsteps):
    stream = torch.cuda.current_stream()
    rc, cur = cue.sim_run_static(
        sim.params, sim.cone, b["fields"][0].data_ptr(), b["fields"][1].data_ptr(), b["src_cell"].data_ptr(),
        b["src_emit"].data_ptr(), b["src_cell"].numel(),
        0 if b["src_map"] is None else b["src_map"].data_ptr(), b["pos"].data_ptr(), b["dir"].data_ptr(),
        b["active"].data_ptr(), b["active"].numel(), step0, nsteps, stream.cuda_stream)
    assert rc == cue.CUE_OK, cue.cue_strerror(rc)
    torch.cuda.synchronize()
    if cur == 1:        # keep the current field in buffer 0 for the next call
        b["fields"][0].copy_(b["fields"][1])
    return b["fields"][0].cpu().numpy()


@pytest.mark.parametrize("name", ["2d-fused", "3d-plain", "2d-map-anysize"])
def test_static_scratch_run_matches_sim_run_twice(cue, name):
    import torch
    if name == "2d-fused":
        w = W.make(name, 2, 300, 212, n_src=9, n_axons=777, C0="smooth", seed=41, stop_radius=2.0)
    elif name == "3d-plain":
        w = W.make(name, 3, 40, 36, 20, dt=0.15, n_src=7, n_axons=500, C0="smooth", seed=42)
    else:
        w = W.make(name, 2, 131, 77, n_src=5, n_axons=300, C0="smooth", seed=43, src_map=True, wall_mode=1)
    ref = cue.Simulation(w)
    b = _buffers(torch, w)
    step = 0
    for nsteps in (13, 21):                      # two calls in a row
        ref.sim_run(nsteps)
        ref.check()
        C = _static_call(cue, torch, ref, b, step, nsteps)
        step += nsteps
        Cr, pr, dr, ar, fs, cs = ref.snapshot()
        assert fs == cs == step
        assert cue.cue_static_status(torch.cuda.current_stream().cuda_stream) == cue.CUE_OK
        # the same initialisation, path choice and kernels on the same state: equal bit for bit
        # (scratch left over from the previous call must not nudge anything)
        np.testing.assert_array_equal(C, Cr)
        np.testing.assert_array_equal(b["pos"].cpu().numpy(), pr)
        np.testing.assert_array_equal(b["dir"].cpu().numpy(), dr)
        np.testing.assert_array_equal(b["active"].cpu().numpy(), ar)
    ref.close()


def test_static_scratch_reports_device_status(cue):
    """A NaN in the field must come back from cue_static_status, and the word must then be clear."""
    import torch
    w = W.make("static-nan", 2, 64, 64, n_src=1, n_axons=4, C0="smooth", seed=44)
    w.C0 = w.C0.copy()
    w.C0[10, 10] = np.nan
    ref = cue.Simulation(w)
    b = _buffers(torch, w)
    stream = torch.cuda.current_stream().cuda_stream
    _static_call(cue, torch, ref, b, 0, 3)
    assert cue.cue_static_status(stream) == cue.CUE_ERR_NONFINITE
    assert cue.cue_static_status(stream) == cue.CUE_OK          # read once, then cleared
    clean = _buffers(torch, W.make("static-ok", 2, 64, 64, n_src=1, n_axons=4, C0="smooth", seed=44))
    _static_call(cue, torch, ref, clean, 3, 2)
    assert cue.cue_static_status(stream) == cue.CUE_OK
    ref.close()


def test_static_scratch_rejects_oversized_problems(cue):
    limit = cue.cue_static_scratch_bytes()
    assert limit == 4 << 20
    big = cue.cue_params(2, 8192, 8192, 1, 1.0, 1.0, 0.01, 0.2, 0)
    assert cue.cue_workspace_bytes(big, 64, 1 << 20) > limit
    cone = cue.cone_params(0.5, 0.4, 0.1, 0.5, 0.0, 1e-15, 0, 0, 1)
    # null buffers: the size check must refuse first; were it ever moved after the argument
    # checks the call would still fail on the host (CUE_ERR_ARG) and queue nothing
    rc, _ = cue.sim_run_static(big, cone, 0, 0, 0, 0, 64, 0, 0, 0, 0, 1 << 20, 0, 1, 0)
    assert rc == cue.CUE_ERR_SCRATCH
