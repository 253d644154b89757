"""The persistent 2D path (one cooperative launch for a whole run, a bounded grid
barrier between steps).

Per node and per cone it computes the plain path's arithmetic in the same
order, so the two must agree bit for bit (source cells are distinct in these
workloads); the tile and grid shape must not change any result; a barrier that
waits for an arrival that never comes must give up, report CUE_ERR_TIMEOUT and
leave the context usable.
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
    if name == "c1-128":
        return W.make(name, 2, 128, 128, n_src=4, n_axons=64, C0="smooth", seed=40)
    if name == "2d-300x212-stop":
        return W.make(name, 2, 300, 212, n_src=9, n_axons=777, C0="smooth", seed=41, stop_radius=2.0)
    if name == "2d-8x8":
        return W.make(name, 2, 8, 8, n_src=2, n_axons=16, C0="random", seed=42)
    if name == "2d-1000x64":
        return W.make(name, 2, 1000, 64, n_src=20, n_axons=3000, C0="smooth", seed=43, stop_radius=3.0)
    if name == "2d-64x1000":
        return W.make(name, 2, 64, 1000, n_src=20, n_axons=3000, C0="smooth", seed=44)
    if name == "map-256x192-clamp":
        return W.make(name, 2, 256, 192, n_src=12, n_axons=1000, C0="smooth", seed=45, src_map="random",
                      wall_mode=1)
    if name == "c5-1024":
        w = W.config_c5()
        w.C0 = W._smooth_field(np.random.default_rng(46), w.shape)
        w.src_map = np.random.default_rng(47).uniform(0, 1, w.shape).astype(np.float32)
        return w
    raise KeyError(name)


def _run(cue, w, path, nsteps, **opts):
    sim = cue.Simulation(w, path=path)
    for k, v in opts.items():
        sim.set_option(getattr(cue, k), v)
    sim.sim_run(nsteps)
    sim.check()
    out = sim.snapshot()
    used = sim.last_path()
    sim.close()
    return out, used


def _assert_same(sa, sb):
    for x, y, what in zip(sa[:4], sb[:4], ("field", "pos", "dir", "active")):
        assert np.array_equal(x, y), f"{what} differs: max {np.abs(x.astype(float) - y.astype(float)).max()}"
    assert sa[4:] == sb[4:]


@pytest.mark.parametrize("name", ["c1-128", "2d-300x212-stop", "2d-8x8", "2d-1000x64", "2d-64x1000",
                                  "map-256x192-clamp", "c5-1024"])
@pytest.mark.parametrize("nsteps", [1, 2, 37])
def test_persist_equals_plain_bitwise(cue, name, nsteps):
    w = _case(name)
    a, pa = _run(cue, w, cue.CUE_PATH_PLAIN, nsteps)
    b, pb = _run(cue, w, cue.CUE_PATH_PERSIST, nsteps)
    assert pa == cue.CUE_PATH_PLAIN and pb == cue.CUE_PATH_PERSIST
    _assert_same(a, b)


@pytest.mark.parametrize("rows,blocks", [(1, 1), (2, 2), (4, 3), (4, 4), (1, 8)])
def test_tile_and_grid_shape_do_not_change_results(cue, rows, blocks):
    w = _case("map-256x192-clamp")
    ref, _ = _run(cue, w, cue.CUE_PATH_PLAIN, 23)
    got, used = _run(cue, w, cue.CUE_PATH_PERSIST, 23, CUE_OPT_PERSIST_ROWS=rows, CUE_OPT_PERSIST_BLOCKS=blocks)
    assert used == cue.CUE_PATH_PERSIST
    _assert_same(ref, got)


def test_auto_takes_the_persistent_path_for_small_grids_beyond_one_block(cue):
    """Grids too small for the fused kernel whose bands do not fit one cluster's shared memory,
    or with more than 128 cones per cluster CTA (where the cluster path measured slower);
    smaller ones run on the cluster or resident paths."""
    for name in ("c5-1024", "2d-1000x64"):
        sim = cue.Simulation(_case(name))
        sim.sim_run(3)
        sim.check()
        assert sim.last_path() == cue.CUE_PATH_PERSIST
        assert sim.get_option(cue.CUE_INFO_GRID) > 0
        sim.close()


def test_one_persistent_step_matches_oracle(cue):
    w = _case("map-256x192-clamp")
    sim = cue.Simulation(w, path=cue.CUE_PATH_PERSIST)
    sim.load(step=91)
    sim.sim_run(1)
    sim.check()
    C1, pos, dirs, act, fs, cs = sim.snapshot()
    assert (fs, cs) == (92, 92)
    C0 = w.field0().astype(np.float64)
    want = oracle.field_step(grid_of(w), C0, w.src_cell, w.src_emit, w.src_map)
    assert field_rel_err(C1, want) <= FIELD_RTOL
    p, d, a = oracle.cone_step(grid_of(w), cone_of(w), C0, 91, w.pos, w.dir, w.active, w.src_cell)
    keep = ~ambiguous_cones(w, C0, 91, w.pos, w.dir, w.active)
    assert (~keep).sum() <= 2
    np.testing.assert_array_equal(act[keep], a[keep])
    assert pos_rel_err(pos[:, keep], p[:, keep]).max() <= POS_RTOL
    assert np.abs(dirs[:, keep] - d[:, keep]).max() <= 1e-5
    sim.close()


def test_barrier_timeout_is_reported_and_the_context_survives(cue):
    """A phantom arrival the barrier waits for never comes: every block gives up after the
    poll limit, the launch ends, the status says CUE_ERR_TIMEOUT; the next run is normal."""
    w = _case("c1-128")
    sim = cue.Simulation(w, path=cue.CUE_PATH_PERSIST)
    sim.set_option(cue.CUE_OPT_WAIT_LIMIT, 4096)
    sim.set_option(cue.CUE_OPT_BARRIER_PHANTOM, 1)
    sim.sim_run(4)
    assert sim.status() == cue.CUE_ERR_TIMEOUT
    assert sim.status() == cue.CUE_OK                   # cleared after reporting
    sim.set_option(cue.CUE_OPT_BARRIER_PHANTOM, 0)
    sim.set_option(cue.CUE_OPT_WAIT_LIMIT, 0)
    sim.load(C=w.field0(), pos=w.pos, dir=w.dir, active=w.active, step=0)
    sim.sim_run(9)
    sim.check()
    got = sim.snapshot()
    sim.close()
    ref, _ = _run(cue, w, cue.CUE_PATH_PLAIN, 9)
    _assert_same(ref, got)


def test_adjoint_recompute_on_the_persistent_path_matches_the_plain_path(cue):
    w = W.config_c5(seed=60, n=64, n_src=2, n_axons=64, nsteps=96)
    out = []
    for path in (cue.CUE_PATH_PLAIN, cue.CUE_PATH_AUTO):
        sim = cue.Simulation(w, path=path)
        g = sim.adjoint(w.targets, 96, 32)
        sim.check()
        out.append({k: v.cpu().numpy() for k, v in g.items() if v is not None})
        sim.close()
    a, b = out
    assert a["loss"] == b["loss"]
    for k in ("dD", "dlambda", "dsrc", "dmap"):
        # identical forward states; the backward's float atomics may sum in another order
        assert np.abs(a[k] - b[k]).max() <= 1e-5 * np.abs(a[k]).max(), k
