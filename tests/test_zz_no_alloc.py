"""sim_run_static: the coupled run for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (code running under another framework's
allocator, hosts that forbid device allocation after start-up); this entry
point takes no workspace and keeps its scratch in a fixed device array inside
the library.  Its results must equal sim_run's on the same state, over two
calls in a row (the second continues where the first stopped, on the scratch
the first call left behind).  The file name keeps it last in collection.
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
        np.testing.assert_allclose(C, Cr, rtol=1e-5, atol=0)
        np.testing.assert_allclose(b["pos"].cpu().numpy(), pr, rtol=1e-5, atol=0)
        np.testing.assert_allclose(b["dir"].cpu().numpy(), dr, rtol=0, atol=1e-5)
        np.testing.assert_array_equal(b["active"].cpu().numpy(), ar)
    ref.close()


def test_static_scratch_rejects_oversized_problems(cue):
    limit = cue.cue_static_scratch_bytes()
    assert limit == 4 << 20
    big = cue.cue_params(2, 8192, 8192, 1, 1.0, 1.0, 0.01, 0.2, 0)
    assert cue.cue_workspace_bytes(big, 64, 1 << 20) > limit
    cone = cue.cone_params(0.5, 0.4, 0.1, 0.5, 0.0, 1e-15, 0, 0, 1)
    rc, _ = cue.sim_run_static(big, cone, 0x1000, 0x2000, 0x3000, 0x3000, 64, 0, 0x4000, 0x4000, 0x4000,
                               1 << 20, 0, 1, 0)
    assert rc == cue.CUE_ERR_SCRATCH
