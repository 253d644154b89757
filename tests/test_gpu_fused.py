"""The fused, temporally blocked 2D path (one launch = K coupled steps).

It computes exactly the plain path's arithmetic in the same order, so the two
must agree bit for bit; it is also compared with the FP64 oracle over whole
K-step blocks.
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
        return W.make(name, 2, 128, 128, n_src=4, n_axons=64, C0="smooth", seed=30)
    if name == "2d-300x212":
        return W.make(name, 2, 300, 212, n_src=9, n_axons=777, C0="smooth", seed=31, stop_radius=2.0)
    if name == "2d-8x8":
        return W.make(name, 2, 8, 8, n_src=2, n_axons=16, C0="random", seed=32)
    if name == "2d-1000x64":
        return W.make(name, 2, 1000, 64, n_src=20, n_axons=3000, C0="smooth", seed=33, stop_radius=3.0)
    if name == "2d-64x1000":
        return W.make(name, 2, 64, 1000, n_src=20, n_axons=3000, C0="smooth", seed=34)
    if name == "c2-2048":
        w = W.config_c2()
        w.C0 = W._smooth_field(np.random.default_rng(35), w.shape)
        return w
    raise KeyError(name)


def _pair(cue, w, K):
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    b = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    b.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, K)
    return a, b


def _assert_same(sa, sb):
    for x, y, what in zip(sa[:4], sb[:4], ("field", "pos", "dir", "active")):
        assert np.array_equal(x, y), f"{what} differs: max {np.abs(x.astype(float) - y.astype(float)).max()}"
    assert sa[4:] == sb[4:]


@pytest.mark.parametrize("name", ["c1-128", "2d-300x212", "2d-8x8", "2d-1000x64", "2d-64x1000"])
@pytest.mark.parametrize("K", [1, 3, 8, 16])
def test_fused_equals_plain_bitwise(cue, name, K):
    w = _case(name)
    a, b = _pair(cue, w, K)
    n = 2 * K + 3                     # two full blocks and a ragged one
    a.sim_run(n)
    b.sim_run(n)
    assert b.fused_active() and not a.fused_active()
    a.check()
    b.check()
    _assert_same(a.snapshot(), b.snapshot())
    assert a.cone_updates() == b.cone_updates()
    a.close()
    b.close()


def test_fused_equals_plain_bitwise_full_c2_size(cue):
    w = _case("c2-2048")
    a, b = _pair(cue, w, 8)
    a.sim_run(20)
    b.sim_run(20)
    _assert_same(a.snapshot(), b.snapshot())
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["c1-128", "2d-300x212"])
def test_fused_field_only_equals_plain(cue, name):
    w = _case(name)
    a, b = _pair(cue, w, 8)
    a.cue_step(11)
    b.cue_step(11)
    assert b.fused_active()
    _assert_same(a.snapshot(), b.snapshot())


def _oracle_block(w, C, step0, K, pos, dirs, act):
    g, c = grid_of(w), cone_of(w)
    amb = np.zeros(act.shape[0], bool)
    C = C.astype(np.float64)
    for j in range(K):
        amb |= ambiguous_cones(w, C, step0 + j, pos, dirs, act)
        pos, dirs, act = oracle.cone_step(g, c, C, step0 + j, pos, dirs, act, w.src_cell)
        C = oracle.field_step(g, C, w.src_cell, w.src_emit, w.src_map)
    return C, pos, dirs, act, amb


@pytest.mark.parametrize("name", ["c1-128", "2d-300x212", "2d-1000x64", "c2-2048"])
def test_fused_single_step_matches_oracle(cue, name):
    """Depth 1: the fused kernel takes one step from an identical state (the per-step bar)."""
    w = _case(name)
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, 1)
    sim.load(step=321)
    C0, pos0, dir0, act0, _, _ = sim.snapshot()
    sim.sim_run(1)
    sim.check()
    assert sim.fused_active()
    C, pos, dirs, act, _, _ = sim.snapshot()
    Cr, pr, dr, ar, amb = _oracle_block(w, C0, 321, 1, pos0, dir0, act0)
    assert field_rel_err(C, Cr) <= FIELD_RTOL
    keep = ~amb
    np.testing.assert_array_equal(act[keep], ar[keep])
    assert pos_rel_err(pos[:, keep], pr[:, keep]).max(initial=0) <= POS_RTOL


@pytest.mark.parametrize("name", ["c1-128", "2d-300x212", "2d-1000x64", "c2-2048"])
def test_fused_block_matches_oracle(cue, name):
    """A whole 8-step block from an identical state.  FP32 rounding differences add up
    over the block, so the budget is K times the per-step tolerance (the per-step bar is
    checked above and the block equals K plain steps bit for bit)."""
    w = _case(name)
    K = 8
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, K)
    sim.load(step=500)
    C0, pos0, dir0, act0, _, _ = sim.snapshot()
    sim.sim_run(K)
    sim.check()
    C, pos, dirs, act, fs, cs = sim.snapshot()
    assert fs == cs == 500 + K
    Cr, pr, dr, ar, amb = _oracle_block(w, C0, 500, K, pos0, dir0, act0)
    assert field_rel_err(C, Cr) <= K * FIELD_RTOL
    keep = ~amb
    assert amb.sum() <= max(2, 0.01 * act0.sum())
    np.testing.assert_array_equal(act[keep], ar[keep])
    assert pos_rel_err(pos[:, keep], pr[:, keep]).max(initial=0) <= K * POS_RTOL


def test_cones_crossing_tile_boundaries(cue):
    """Cones start on and next to tile edges and run across them for several blocks."""
    w = _case("2d-1000x64")
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.set_option(cue.CUE_OPT_TEMPORAL_DEPTH, 8)
    sim.sim_run(1)
    tile = sim.get_option(cue.CUE_INFO_TILE)
    TX, TY = tile & 0xFFFF, tile >> 16
    assert TX > 0 and TY > 0
    n = w.n_axons
    rng = np.random.default_rng(36)
    edges = np.arange(TX, w.nx - 1, TX, dtype=np.float64)
    px = rng.choice(edges, n) + rng.choice([-1e-3, 0.0, 1e-3, -0.49, 0.49], n)
    py = rng.uniform(1, w.ny - 2, n)
    pos = np.stack([px, py]).astype(np.float32)
    d = np.stack([rng.choice([-1.0, 1.0], n), np.zeros(n)]).astype(np.float32)
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    for s in (a, sim):
        s.load(C=w.field0(), pos=pos, dir=d, active=np.ones(n, np.uint8), step=0)
        s.sim_run(29)
    _assert_same(a.snapshot(), sim.snapshot())


def test_all_cones_in_one_tile(cue):
    w = _case("c1-128")
    n = 5000
    rng = np.random.default_rng(37)
    w.pos = rng.uniform(60, 62, (2, n)).astype(np.float32)
    w.dir = W._directions(rng, 2, n).astype(np.float32)
    w.active = np.ones(n, np.uint8)
    a, b = _pair(cue, w, 8)
    a.sim_run(17)
    b.sim_run(17)
    _assert_same(a.snapshot(), b.snapshot())


def test_clustered_workload_equals_plain(cue):
    """The clustered 2048^2 workload (16,384 cones in four 48 x 48 squares, wall clamp): every
    crowded tile steps its overflow cones from global memory; three fused launches and a ragged
    fourth equal the plain path bit for bit."""
    w = W.config_c2_clustered()
    a, b = _pair(cue, w, 8)
    a.sim_run(29)
    b.sim_run(29)
    _assert_same(a.snapshot(), b.snapshot())


def test_clustered_cones_spill_path_on_a_large_grid(cue):
    """A grid large enough that per-tile bins holding every cone would pass the workspace
    budget (4096^2, 8,448 cones): bins hold 512 ids and the rest of a crowded tile's cones go
    to the spill list.  5,000 cones start in one tile and 3,448 spread over the grid; both
    runs must equal the plain path bit for bit."""
    w = W.make("spill-4096", 2, 4096, 4096, n_src=16, n_axons=8448, C0="smooth", seed=39, stop_radius=2.0)
    rng = np.random.default_rng(39)
    w.pos[:, :5000] = rng.uniform(1000, 1040, (2, 5000)).astype(np.float32)
    a, b = _pair(cue, w, 8)
    a.sim_run(19)
    b.sim_run(19)
    _assert_same(a.snapshot(), b.snapshot())


def test_fused_unsupported_shapes_are_refused(cue):
    w = W.make("odd", 2, 257, 131, n_src=3, n_axons=10, C0="smooth", seed=38)
    sim = cue.Simulation(w)
    with pytest.raises(cue.CueError):
        sim.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_FUSED)
    sim.sim_run(3)               # auto: falls back to the plain kernels
    assert not sim.fused_active()
    sim.check()


def test_fused_reports_nonfinite(cue):
    w = _case("2d-300x212")
    w.C0 = w.field0()
    w.C0[100, 150] = np.inf
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.sim_run(8)
    assert sim.status() == cue.CUE_ERR_NONFINITE


def _run_twice_with_helpers(cue, w, n, K=8):
    """Two runs on each path: the fused handle's second run takes the helper count the
    first run's crowding reported (its readback has landed after the synchronize)."""
    import torch
    a, b = _pair(cue, w, K)
    a.sim_run(n)
    b.sim_run(n)
    torch.cuda.synchronize()
    assert b.get_option(cue.CUE_INFO_HELPERS) == 0          # nothing reported before the first run
    a.sim_run(n)
    b.sim_run(n)
    helpers = b.get_option(cue.CUE_INFO_HELPERS)
    a.check()
    b.check()
    _assert_same(a.snapshot(), b.snapshot())
    assert a.cone_updates() == b.cone_updates()
    a.close()
    b.close()
    return helpers


def test_clustered_workload_with_helpers_equals_plain(cue):
    """The clustered 2048^2 workload: the second run shares each crowded tile's cones out
    to helper blocks (192 per block, the cone warps' register slots) and must still equal the plain path bit for bit."""
    helpers = _run_twice_with_helpers(cue, W.config_c2_clustered(), 21)
    assert helpers > 0


def test_helpers_all_cones_in_one_tile(cue):
    w = _case("c1-128")
    n = 5000
    rng = np.random.default_rng(40)
    w.pos = rng.uniform(60, 62, (2, n)).astype(np.float32)
    w.dir = W._directions(rng, 2, n).astype(np.float32)
    w.active = np.ones(n, np.uint8)
    assert _run_twice_with_helpers(cue, w, 17) >= 10


def test_helpers_fewer_than_needed(cue):
    """60,000 cones in one tile need 312 helpers, more than the 128 a launch takes: the
    tile's own block steps the cones past the helpers' slices."""
    w = W.make("crowd-1024", 2, 1024, 512, n_src=8, n_axons=60000, C0="smooth", seed=41, wall_mode=1)
    rng = np.random.default_rng(41)
    w.pos = rng.uniform(300, 340, (2, 60000)).astype(np.float32)
    assert _run_twice_with_helpers(cue, w, 9) == 128


def test_uniform_workload_takes_no_helpers(cue):
    import torch
    w = _case("c2-2048")
    sim = cue.Simulation(w, path=cue.CUE_PATH_FUSED)
    sim.sim_run(16)
    torch.cuda.synchronize()
    sim.sim_run(16)
    assert sim.get_option(cue.CUE_INFO_HELPERS) == 0
    sim.close()


def test_many_sources_spread_out_run_fused(cue):
    """1,500 point sources in total, none of the tile regions holding more than its list's
    256: the fused path takes them and equals the plain path bit for bit."""
    w = W.make("src-1500", 2, 1024, 768, n_src=1500, n_axons=2000, C0="smooth", seed=42, stop_radius=1.5)
    a, b = _pair(cue, w, 8)
    a.sim_run(19)
    b.sim_run(19)
    assert b.fused_active()
    _assert_same(a.snapshot(), b.snapshot())
    a.close()
    b.close()


def test_sources_crowding_one_tile_are_refused(cue):
    """300 sources inside one tile's region exceed its list: the fused path is refused and
    AUTO runs the plain kernels."""
    w = W.make("src-crowd", 2, 1024, 768, n_src=300, n_axons=100, C0="smooth", seed=43)
    rng = np.random.default_rng(43)
    xs = rng.choice(60, 300, replace=True) + 100
    ys = rng.choice(40, 300, replace=True) + 100
    cells = np.unique(ys * w.nx + xs).astype(np.int32)
    while cells.size < 300:                                  # distinct cells in a 60 x 40 block
        extra = (rng.integers(100, 140) * w.nx + rng.integers(100, 160))
        cells = np.unique(np.append(cells, extra)).astype(np.int32)
    w.src_cell = cells[:300]
    sim = cue.Simulation(w)
    with pytest.raises(cue.CueError):
        sim.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_FUSED)
    sim.sim_run(3)
    assert not sim.fused_active()
    sim.check()
    sim.close()


def test_helpers_with_cones_stopping_at_sources(cue):
    """A crowded tile whose cones stop at nearby sources as they go: helper slices step and
    re-bin only the cones still moving, and the run equals the plain path bit for bit."""
    w = W.make("crowd-stop", 2, 1024, 512, n_src=12, n_axons=6000, C0="smooth", seed=44, stop_radius=3.0)
    rng = np.random.default_rng(44)
    w.pos = rng.uniform(300, 360, (2, 6000)).astype(np.float32)
    cells = np.unique(rng.integers(310, 350, 12) * w.nx + rng.integers(310, 350, 12)).astype(np.int32)
    w.src_cell = cells
    w.src_emit = np.ones(cells.size, np.float32)
    helpers = _run_twice_with_helpers(cue, w, 13)
    assert helpers > 0
