"""GPU (FP32, through the C ABI) vs FP64 oracle, one step from identical state.

Sizes span several thread blocks with ragged tails, the vectorised and the
any-size kernels, and the full benchmark grids (2D 2048^2 with 16,384 cones,
3D 256^3 with 65,536 cones).  Tolerances are in tests/parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1405_3331_gb300 import workloads as W
from parity import (FIELD_RTOL, POS_RTOL, ambiguous_cones, cone_of, field_rel_err, grid_of,
                    pos_rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cue():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


def _case(name):
    if name == "c1-128":
        return W.make(name, 2, 128, 128, lam=0.01, n_src=4, n_axons=64, C0="smooth", seed=10)
    if name == "2d-300x212":
        return W.make(name, 2, 300, 212, n_src=9, n_axons=777, C0="smooth", seed=11,
                      stop_radius=2.0)
    if name == "2d-257x131-anysize":
        return W.make(name, 2, 257, 131, n_src=5, n_axons=333, C0="smooth", seed=12)
    if name == "2d-2x2":
        return W.make(name, 2, 2, 2, n_src=1, n_axons=5, C0="random", seed=13)
    if name == "2d-6x3":
        return W.make(name, 2, 6, 3, n_src=2, n_axons=9, C0="random", seed=14)
    if name == "3d-40x36x20":
        return W.make(name, 3, 40, 36, 20, dt=0.15, n_src=7, n_axons=500, C0="smooth", seed=15,
                      stop_radius=2.0)
    if name == "3d-33x17x9-anysize":
        return W.make(name, 3, 33, 17, 9, dt=0.15, n_src=3, n_axons=200, C0="smooth", seed=16)
    if name == "c5-map-1024-clamp":
        return W.make(name, 2, 1024, 1024, n_src=32, n_axons=4096, C0="smooth", seed=17,
                      src_map="random", wall_mode=1)
    if name == "c2-2048":
        w = W.config_c2()
        w.C0 = W._smooth_field(np.random.default_rng(18), w.shape)
        return w
    if name == "c3-256":
        w = W.config_c3()
        w.C0 = np.random.default_rng(19).uniform(0, 1, w.shape).astype(np.float32)
        return w
    raise KeyError(name)


CASES = ["c1-128", "2d-300x212", "2d-257x131-anysize", "2d-2x2", "2d-6x3", "3d-40x36x20",
         "3d-33x17x9-anysize", "c5-map-1024-clamp", "c2-2048", "c3-256"]


def _sim(cue, w, step=0):
    sim = cue.Simulation(w)
    if step:
        sim.load(step=step)
    return sim


@pytest.mark.parametrize("name", CASES)
def test_field_step_matches_oracle(cue, name):
    w = _case(name)
    sim = _sim(cue, w)
    C0 = w.field0()
    sim.cue_step(1)
    sim.check()
    got = sim.field().cpu().numpy()
    want = oracle.field_step(grid_of(w), C0.astype(np.float64), w.src_cell, w.src_emit, w.src_map)
    err = field_rel_err(got, want)
    assert err <= FIELD_RTOL, err
    sim.close()


def _compare_cones(w, C, step, pos0, dir0, act0, got_pos, got_dir, got_act):
    want_pos, want_dir, want_act = oracle.cone_step(grid_of(w), cone_of(w), C.astype(np.float64), step,
                                                    pos0, dir0, act0, w.src_cell)
    amb = ambiguous_cones(w, C.astype(np.float64), step, pos0, dir0, act0)
    keep = ~amb
    assert amb.sum() <= max(2, 0.01 * act0.sum()), amb.sum()
    np.testing.assert_array_equal(got_act[keep], want_act[keep])
    err = pos_rel_err(got_pos[:, keep], want_pos[:, keep])
    assert (err.max() if err.size else 0.0) <= POS_RTOL, err.max()
    derr = np.abs(got_dir[:, keep] - want_dir[:, keep]).max() if keep.any() else 0.0
    assert derr <= 1e-5, derr
    return int(amb.sum())


@pytest.mark.parametrize("name", CASES)
def test_cone_step_matches_oracle(cue, name):
    w = _case(name)
    step = 1234
    sim = _sim(cue, w, step=step)
    C0 = w.field0()
    sim.cone_step(1)
    sim.check()
    _, pos, dirs, act, fs, cs = sim.snapshot()
    assert (fs, cs) == (step, step + 1)
    _compare_cones(w, C0, step, w.pos, w.dir, w.active, pos, dirs, act)
    sim.close()


@pytest.mark.parametrize("name", ["c1-128", "2d-300x212", "3d-40x36x20", "c5-map-1024-clamp", "c2-2048"])
def test_sim_run_one_step_matches_oracle(cue, name):
    w = _case(name)
    sim = _sim(cue, w, step=77)
    C0 = w.field0()
    sim.sim_run(1)
    sim.check()
    C1, pos, dirs, act, fs, cs = sim.snapshot()
    assert (fs, cs) == (78, 78)
    want = oracle.field_step(grid_of(w), C0.astype(np.float64), w.src_cell, w.src_emit, w.src_map)
    assert field_rel_err(C1, want) <= FIELD_RTOL
    _compare_cones(w, C0, 77, w.pos, w.dir, w.active, pos, dirs, act)
    sim.close()


@pytest.mark.parametrize("name,after", [("c1", 1), ("c1", 10), ("c1", 100), ("c1", 499)])
def test_per_step_parity_along_a_run(cue, name, after):
    """Run the GPU `after` steps from C0 = 0, copy its state into the oracle, step both once."""
    w = W.config_c1()
    sim = _sim(cue, w)
    sim.sim_run(after)
    sim.check()
    C, pos, dirs, act, fs, cs = sim.snapshot()
    assert fs == cs == after
    sim.sim_run(1)
    sim.check()
    C1, pos1, dirs1, act1, _, _ = sim.snapshot()
    want = oracle.field_step(grid_of(w), C.astype(np.float64), w.src_cell, w.src_emit)
    assert field_rel_err(C1, want) <= FIELD_RTOL
    _compare_cones(w, C, after, pos, dirs, act, pos1, dirs1, act1)
    sim.close()


def test_cone_then_field_is_sim_run_bitwise(cue):
    w = _case("2d-300x212")
    a = _sim(cue, w)
    b = _sim(cue, w)
    for _ in range(5):
        a.cone_step(1)
        a.cue_step(1)
    b.sim_run(5)
    sa, sb = a.snapshot(), b.snapshot()
    for x, y in zip(sa[:4], sb[:4]):
        np.testing.assert_array_equal(x, y)
    assert sa[4:] == sb[4:] == (5, 5)


def test_noise_direction_matches_oracle(cue):
    """w_prev = w_grad = 0: the new direction is xi/|xi|, exposing the Philox/Box-Muller path."""
    for dim in (2, 3):
        w = W.make("noise", dim, 64, 64, 64 if dim == 3 else 1, dt=0.15, n_src=0, n_axons=4096,
                   w=(0.0, 0.0, 1.0), step_len=0.01, seed=20)
        sim = _sim(cue, w, step=99)
        sim.cone_step(1)
        _, _, dirs, act, _, _ = sim.snapshot()
        xi = oracle.noise(w.seed, np.arange(4096), 99, dim)[:, :dim]
        want = xi / np.linalg.norm(xi, axis=1, keepdims=True)
        moved = act.astype(bool)          # cones that left the domain keep their direction
        assert moved.sum() > 4000
        assert np.abs(dirs.T[moved] - want[moved]).max() < 2e-6
        sim.close()


def test_empty_inputs(cue):
    w = W.make("empty", 2, 64, 32, n_src=0, n_axons=0, C0="smooth", seed=21)
    sim = _sim(cue, w)
    sim.sim_run(3)
    sim.check()
    C = sim.field().cpu().numpy()
    want, *_ = oracle.run(grid_of(w), cone_of(w), w.field0(), 0, 3)
    assert field_rel_err(C, want) <= FIELD_RTOL
    sim.sim_run(0)
    assert sim.state() == (3, 3, 1)
    sim.close()


def test_out_of_range_source_is_reported_and_skipped(cue):
    w = W.make("bounds", 2, 64, 64, n_src=3, n_axons=8, C0="smooth", seed=22)
    w.src_cell = np.array([5, 64 * 64 + 7, -3], np.int32)
    sim = _sim(cue, w)
    assert sim.status() == cue.CUE_ERR_BOUNDS   # the source-coordinate pass already saw them
    sim.cue_step(1)
    assert sim.status() == cue.CUE_ERR_BOUNDS
    assert sim.status() == cue.CUE_OK          # cleared after reporting
    got = sim.field().cpu().numpy()
    want = oracle.field_step(grid_of(w), w.field0().astype(np.float64), [5], w.src_emit[:1])
    assert field_rel_err(got, want) <= FIELD_RTOL
    sim.close()


def test_nonfinite_is_reported(cue):
    w = W.make("nan", 2, 64, 64, n_src=1, n_axons=4, C0="smooth", seed=23)
    w.C0 = w.field0()
    w.C0[10, 10] = np.nan
    sim = _sim(cue, w)
    sim.cue_step(1)
    assert sim.status() == cue.CUE_ERR_NONFINITE
    sim.close()


def test_call_order_is_enforced(cue):
    w = _case("c1-128")
    sim = _sim(cue, w)
    sim.cone_step(1)
    with pytest.raises(cue.CueError) as e:
        sim.sim_run(1)
    assert e.value.code == cue.CUE_ERR_STATE
    sim.cue_step(1)
    sim.sim_run(1)          # counters agree again
    sim.check()
    sim.close()


def test_whole_run_field_error_and_endpoint_statistics(cue, record_property):
    """The full 500-step 128^2 run: FP32 field vs FP64 (reported), and endpoint statistics.

    The field does not depend on the cones, so its FP32-vs-FP64 error is a plain accumulated
    rounding error; trajectories are compared as distributions only."""
    import scipy.stats
    w = W.config_c1()
    sim = _sim(cue, w)
    sim.sim_run(w.nsteps)
    sim.check()
    C, pos, dirs, act, _, _ = sim.snapshot()
    Cr, posr, dirr, actr = oracle.run(grid_of(w), cone_of(w), w.field0(), 0, w.nsteps, w.src_cell,
                                      w.src_emit, None, w.pos, w.dir, w.active)
    ferr = field_rel_err(C, Cr)
    record_property("fp32_vs_fp64_field_rel_err_500_steps", ferr)
    assert ferr < 1e-4
    disp_gpu = np.linalg.norm(pos - w.pos, axis=0)
    disp_ref = np.linalg.norm(posr - w.pos, axis=0)
    ks = scipy.stats.ks_2samp(disp_gpu, disp_ref).pvalue
    record_property("endpoint_displacement_ks_pvalue", ks)
    record_property("endpoint_identical_fraction", float(np.mean(pos_rel_err(pos, posr) < 1e-4)))
    assert ks > 1e-3


@pytest.mark.parametrize("name", ["2d-300x212", "3d-40x36x20", "c3-256"])
def test_vector_and_tma_field_kernels_equal_the_any_size_kernel(cue, name):
    """Aligned buffers run the float4 / TMA kernels, a one-float offset the any-size
    kernel; all evaluate the same node-update expression, so the fields agree bit for bit."""
    w = _case(name)
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    b = cue.Simulation(w, path=cue.CUE_PATH_PLAIN, field_offset=1)
    a.cue_step(3)
    b.cue_step(3)
    a.check()
    b.check()
    np.testing.assert_array_equal(a.field().cpu().numpy(), b.field().cpu().numpy())
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["3d-40x36x20", "c3-256"])
def test_merged_3d_step_equals_separate_launches(cue, name):
    """With the TMA field kernel a 3D step (cones, field, sources) is one launch (each field
    block steps a slice of the cones while its first planes load); with a one-float offset
    it is three.  Same arithmetic in the same order: the whole state
    agrees bit for bit after several steps (sources sit on distinct nodes)."""
    w = _case(name)
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    b = cue.Simulation(w, path=cue.CUE_PATH_PLAIN, field_offset=1)
    l0a, l0b = a.launches(), b.launches()
    a.sim_run(4)
    b.sim_run(4)
    a.check()
    b.check()
    assert a.launches() - l0a == 4
    assert b.launches() - l0b == 12
    for x, y in zip(a.snapshot()[:4], b.snapshot()[:4]):
        np.testing.assert_array_equal(x, y)
    a.close()
    b.close()
