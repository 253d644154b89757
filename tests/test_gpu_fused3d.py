"""The temporally blocked 3D path (one launch = two coupled steps).

It evaluates the one-launch-per-step 3D kernels' arithmetic in the same
order, so the two paths must agree bit for bit (field, cone state, stop flags
and cone-update counts) over runs with odd and even step counts; it is also
held to the FP64 oracle over one launch from an identical state.  Cases cover
cones crowded past the shared-memory slots of a box, the source-stop radius,
the wall clamp, a dense rate map, walls on every side, the field-only call and
the full 256^3 workload.
"""
import numpy as np
import pytest

import oracle
from paper_1405_3331_gb300 import workloads as W
from parity import FIELD_RTOL, POS_RTOL, ambiguous_cones, cone_of, field_rel_err, grid_of, pos_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cue():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


def _case(name):
    if name == "3d-40x36x20":
        return W.make(name, 3, 40, 36, 20, dt=0.15, n_src=7, n_axons=500, C0="smooth", seed=70)
    if name == "3d-136x40x30-map":
        return W.make(name, 3, 136, 40, 30, dt=0.15, n_src=9, n_axons=900, C0="smooth", seed=71, src_map=True)
    if name == "3d-64x48x40-stop":
        return W.make(name, 3, 64, 48, 40, dt=0.15, n_src=12, n_axons=2000, C0="smooth", seed=72, stop_radius=2.5)
    if name == "3d-64x48x40-clamp":
        return W.make(name, 3, 64, 48, 40, dt=0.15, n_src=5, n_axons=1500, C0="smooth", seed=73, wall_mode=1)
    if name == "3d-crowd":
        # 3,000 of 3,500 cones in one box: past the shared-memory slots, the rest from global memory
        w = W.make(name, 3, 64, 48, 40, dt=0.15, n_src=6, n_axons=3500, C0="smooth", seed=74)
        rng = np.random.default_rng(74)
        w.pos[:2, :3000] = rng.uniform(4.0, 12.0, (2, 3000)).astype(np.float32)
        w.pos[2, :3000] = rng.uniform(5.1, 5.9, 3000).astype(np.float32)
        return w
    if name == "3d-260x30x9-walls":
        # cones on every wall, edge and corner (wall clamp keeps them there)
        w = W.make(name, 3, 260, 30, 9, dt=0.15, n_src=4, n_axons=600, C0="random", seed=75, wall_mode=1)
        rng = np.random.default_rng(75)
        hi = np.array([259.0, 29.0, 8.0])[:, None]
        corner = rng.integers(0, 2, (3, 600)) * hi
        pick = rng.integers(0, 3, 600)
        mix = w.pos.astype(np.float64).copy()
        for ax in range(3):
            on = pick != ax
            mix[ax, on] = corner[ax, on]
        w.pos = mix.astype(np.float32)
        return w
    if name == "c3-256":
        w = W.config_c3()
        w.C0 = W._smooth_field(np.random.default_rng(76), w.shape)
        return w
    raise KeyError(name)


def _pair(cue, w):
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    b = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    return a, b


def _assert_same(sa, sb):
    for x, y, what in zip(sa[:4], sb[:4], ("field", "pos", "dir", "active")):
        assert np.array_equal(x, y), f"{what} differs: max {np.abs(x.astype(float) - y.astype(float)).max()}"
    assert sa[4:] == sb[4:]


CASES = ["3d-40x36x20", "3d-136x40x30-map", "3d-64x48x40-stop", "3d-64x48x40-clamp", "3d-crowd",
         "3d-260x30x9-walls"]


@pytest.mark.parametrize("name", CASES)
def test_blocked_3d_equals_one_step_launches_bitwise(cue, name):
    w = _case(name)
    a, b = _pair(cue, w)
    for n in (7, 6):                  # three launches and an odd last step, then three more
        a.sim_run(n)
        b.sim_run(n)
        assert b.fused_active() and not a.fused_active()
        a.check()
        b.check()
        _assert_same(a.snapshot(), b.snapshot())
    assert a.cone_updates() == b.cone_updates()
    assert b.get_option(cue.CUE_INFO_DEPTH) == 2
    if name == "3d-64x48x40-stop":
        act = b.snapshot()[3]
        assert 0 < int(act.sum()) < w.n_axons          # some cones stopped, some still move
    a.close()
    b.close()


def test_blocked_3d_full_c3_size(cue):
    w = _case("c3-256")
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    b = cue.Simulation(w)
    b.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, 2)        # AUTO with depth 2 takes the blocked path
    a.sim_run(20)
    b.sim_run(20)
    assert b.fused_active()
    tile = b.get_option(cue.CUE_INFO_TILE)
    assert tile & 0xFFFF == 128 and 8 <= tile >> 16 <= 16
    _assert_same(a.snapshot(), b.snapshot())
    assert a.cone_updates() == b.cone_updates()
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["3d-40x36x20", "3d-136x40x30-map"])
def test_blocked_3d_field_only_equals_one_step_launches(cue, name):
    w = _case(name)
    a, b = _pair(cue, w)
    a.cue_step(9)
    b.cue_step(9)
    assert b.fused_active()
    _assert_same(a.snapshot(), b.snapshot())


@pytest.mark.parametrize("name", ["3d-40x36x20", "3d-64x48x40-stop", "3d-136x40x30-map", "c3-256"])
def test_blocked_3d_launch_matches_oracle(cue, name):
    """One launch (two coupled steps) from an identical state against the FP64 oracle's two
    steps; the per-step budget twice over, cones whose decisions rounding may flip excluded."""
    w = _case(name)
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.load(step=401)
    C0, pos0, dir0, act0, _, _ = sim.snapshot()
    sim.sim_run(2)
    sim.check()
    assert sim.fused_active()
    C, pos, dirs, act, fs, cs = sim.snapshot()
    assert fs == cs == 403
    g, c = grid_of(w), cone_of(w)
    Cr = C0.astype(np.float64)
    pr, dr, ar = pos0, dir0, act0
    amb = np.zeros(w.n_axons, bool)
    for j in range(2):
        amb |= ambiguous_cones(w, Cr, 401 + j, pr, dr, ar)
        pr, dr, ar = oracle.cone_step(g, c, Cr, 401 + j, pr, dr, ar, w.src_cell)
        Cr = oracle.field_step(g, Cr, w.src_cell, w.src_emit, w.src_map)
    assert field_rel_err(C, Cr) <= 2 * FIELD_RTOL
    keep = ~amb
    assert amb.sum() <= max(2, 0.01 * act0.sum())
    np.testing.assert_array_equal(act[keep], ar[keep])
    assert pos_rel_err(pos[:, keep], pr[:, keep]).max(initial=0) <= 2 * POS_RTOL
    sim.close()


def test_blocked_3d_reports_nonfinite(cue):
    w = _case("3d-40x36x20")
    w.C0 = w.field0()
    w.C0[10, 18, 20] = np.inf
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.sim_run(2)
    assert sim.status() == cue.CUE_ERR_NONFINITE
    sim.close()


def test_auto_keeps_the_step_kernel(cue):
    """AUTO on a 3D handle runs one launch per step (measured faster on GB300); a temporal
    depth of 2 or CUE_PATH_FUSED selects the blocked path."""
    w = _case("3d-40x36x20")
    a = cue.Simulation(w)
    a.sim_run(4)
    assert not a.fused_active()
    a.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, 2)
    a.sim_run(4)
    assert a.fused_active()
    a.close()


def test_blocked_3d_crowded_box_with_stops(cue):
    """3,000 cones in one box (past its 512 shared-memory slots) around sources with a stop
    radius: cones stop in both sub-steps, in shared memory and in global memory."""
    w = W.make("3d-crowd-stop", 3, 64, 48, 40, dt=0.15, n_src=8, n_axons=3500, C0="smooth", seed=77,
               stop_radius=1.5)
    rng = np.random.default_rng(77)
    w.pos[:2, :3000] = rng.uniform(4.0, 12.0, (2, 3000)).astype(np.float32)
    w.pos[2, :3000] = rng.uniform(5.1, 5.9, 3000).astype(np.float32)
    xs, ys, zs = rng.integers(5, 12, 8), rng.integers(5, 12, 8), rng.integers(4, 8, 8)
    w.src_cell = np.unique((zs * w.ny + ys) * w.nx + xs).astype(np.int32)
    w.src_emit = np.ones(w.src_cell.size, np.float32)
    a, b = _pair(cue, w)
    for n in (6, 9):
        a.sim_run(n)
        b.sim_run(n)
        a.check()
        b.check()
        _assert_same(a.snapshot(), b.snapshot())
    assert a.cone_updates() == b.cone_updates()
    assert int(b.snapshot()[3].sum()) < w.n_axons                 # some cones stopped
    a.close()
    b.close()
