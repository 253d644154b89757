"""Batched runs (include/cue_batch.h): independent 2D instances of uneven sizes and
parameters stepped by one persistent launch.

Each instance must evolve bit for bit as it does alone on the plain path (same
arithmetic per node and per cone, source cells distinct), whatever its nx (the
batch stores rows with a pitch rounded up to 4 and walls can fall inside a
float4), whether the launch is direct or a replayed CUDA graph, and after the
autotuner has measured its candidates (it must restore the state it found).
"""
import numpy as np
import pytest

import oracle
from paper_1405_3331_gb300 import workloads as W
from parity import FIELD_RTOL, compare_cones, field_rel_err, grid_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cue():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


@pytest.fixture(scope="module")
def batch_mod(cue):
    from paper_1405_3331_gb300 import batch
    return batch


def _mixed():
    """Uneven sizes (nx % 4 in {0, 1, 2, 3}), physics, sources, cones, stop and clamp modes."""
    out = [
        W.make("b0", 2, 66, 70, D=0.8, lam=0.02, dt=0.2, n_src=3, n_axons=40, C0="smooth", seed=70),
        W.make("b1", 2, 97, 64, D=1.5, lam=0.001, dt=0.12, n_src=5, n_axons=300, C0="smooth", seed=71,
               stop_radius=2.0),
        W.make("b2", 2, 128, 129, D=1.0, lam=0.05, dt=0.2, n_src=4, n_axons=257, C0="random", seed=72,
               wall_mode=1),
        W.make("b3", 2, 203, 51, D=0.6, lam=0.01, dt=0.3, n_src=8, n_axons=600, C0="smooth", seed=73,
               src_map="random"),
        W.make("b4", 2, 255, 255, D=2.0, lam=0.003, dt=0.1, n_src=16, n_axons=1000, C0="smooth", seed=74,
               stop_radius=3.0),
        W.make("b5", 2, 8, 9, n_src=1, n_axons=3, C0="random", seed=75),
        W.make("b6", 2, 64, 64, n_src=0, n_axons=0, C0="smooth", seed=76),
    ]
    return out


def _alone(cue, w, nsteps):
    sim = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    sim.sim_run(nsteps)
    sim.check()
    C, pos, dirs, act, _, _ = sim.snapshot()
    sim.close()
    return C, pos, dirs, act


def _assert_same(a, b, tag):
    for x, y, what in zip(a, b, ("field", "pos", "dir", "active")):
        assert np.array_equal(x, y), f"{tag}: {what} differs, max {np.abs(x.astype(float) - y.astype(float)).max()}"


@pytest.mark.parametrize("nsteps", [1, 5, 33])
def test_batch_equals_each_instance_alone(cue, batch_mod, nsteps):
    ws = _mixed()
    b = batch_mod.Batch(ws)
    b.run(nsteps)
    b.check()
    for i, w in enumerate(ws):
        _assert_same(b.snapshot(i), _alone(cue, w, nsteps), w.name)
    assert b.get_option(batch_mod.CUE_BINFO_STEP) == nsteps
    b.close()


@pytest.mark.parametrize("rows,blocks,mode,depth", [(1, 1, 1, 0), (2, 3, 1, 0), (4, 2, 1, 0), (1, 0, 2, 0),
                                                    (2, 0, 2, 0), (4, 0, 2, 0), (8, 0, 2, 0), (16, 0, 2, 0),
                                                    (0, 0, 3, 1), (0, 0, 3, 2), (0, 0, 3, 3), (0, 0, 3, 4),
                                                    (0, 0, 3, 5), (0, 0, 3, 8)])
def test_launch_shape_does_not_change_results(cue, batch_mod, rows, blocks, mode, depth):
    """Persistent launches of any shape, one launch per step, and temporally blocked launches
    of any depth (12 steps: ragged last launches for depths 5 and 8) give every instance
    exactly the state it reaches alone on the plain path, and the same cone-update count."""
    ws = _mixed()
    b = batch_mod.Batch(ws)
    assert b.get_option(batch_mod.CUE_BINFO_BLOCKED) == 1
    if rows:
        b.set_option(batch_mod.CUE_BOPT_ROWS, rows)
    b.set_option(batch_mod.CUE_BOPT_BLOCKS, blocks)
    b.set_option(batch_mod.CUE_BOPT_MODE, mode)
    if depth:
        b.set_option(batch_mod.CUE_BOPT_DEPTH, depth)
    b.run(12)
    b.check()
    if rows:
        assert b.get_option(batch_mod.CUE_BOPT_ROWS) == rows
    assert b.get_option(batch_mod.CUE_BOPT_MODE) == mode
    if depth:
        assert b.get_option(batch_mod.CUE_BOPT_DEPTH) == depth
    updates = b.cone_updates()
    want_updates = 0
    for i, w in enumerate(ws):
        alone = _alone(cue, w, 12)
        _assert_same(b.snapshot(i), alone, w.name)
    ref = batch_mod.Batch(ws)
    ref.set_option(batch_mod.CUE_BOPT_MODE, 1)
    ref.run(12)
    want_updates = ref.cone_updates()
    ref.close()
    assert updates == want_updates
    b.close()


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_graph_replays_equal_direct_launches(cue, batch_mod, mode):
    ws = _mixed()
    a = batch_mod.Batch(ws)
    a.run(30)
    g = batch_mod.Batch(ws)
    g.set_option(batch_mod.CUE_BOPT_MODE, mode)
    g.set_option(batch_mod.CUE_BOPT_GRAPH, 1)
    for _ in range(3):
        g.run(10)                                  # captured once, replayed twice
    a.check()
    g.check()
    assert g.get_option(batch_mod.CUE_BOPT_GRAPH) == 1
    for i, w in enumerate(ws):
        _assert_same(a.snapshot(i), g.snapshot(i), w.name)
    a.close()
    g.close()


def test_autotune_restores_the_state_and_keeps_a_valid_shape(cue, batch_mod):
    ws = _mixed()
    b = batch_mod.Batch(ws)
    b.run(3)
    before = [b.snapshot(i) for i in range(len(ws))]
    updates_before = b.cone_updates()
    rows, blocks, ms = b.autotune(8)
    mode = b.get_option(batch_mod.CUE_BOPT_MODE)
    assert ms > 0 and 0 <= blocks <= 8
    if mode == 3:
        assert rows == 0 and blocks == 0 and b.get_option(batch_mod.CUE_BOPT_DEPTH) in (2, 4, 8)
    else:
        assert rows in (1, 2, 4, 8, 16) and mode == (2 if blocks == 0 else 1)
    assert b.get_option(batch_mod.CUE_BINFO_STEP) == 3
    for i in range(len(ws)):
        _assert_same(b.snapshot(i), before[i], ws[i].name)
    assert b.cone_updates() == 0                    # the probes' updates were taken back
    b.run(9)
    b.check()
    for i, w in enumerate(ws):
        _assert_same(b.snapshot(i), _alone(cue, w, 12), w.name)
    assert updates_before > 0
    b.close()


@pytest.mark.parametrize("mode", [1, 3])
def test_batched_workload_sample_equals_instances_alone(cue, batch_mod, mode):
    """Sixteen instances of the 512-instance batched workload (sides U{64..1024}, D ~ U[0.5, 2],
    lambda log-uniform, dt = 0.2 / D, 4-64 sources, 256-4096 cones), persistent and
    temporally blocked (depth 4: two launches)."""
    ws = W.config_c4(n_instances=16, nsteps=8)
    b = batch_mod.Batch(ws)
    b.set_option(batch_mod.CUE_BOPT_MODE, mode)
    b.run(8)
    b.check()
    for i, w in enumerate(ws):
        _assert_same(b.snapshot(i), _alone(cue, w, 8), w.name)
    b.close()


@pytest.mark.parametrize("mode", [2, 3])
def test_long_per_step_runs_replay_a_bounded_graph(cue, batch_mod, mode):
    """A per-step or blocked run longer than one captured graph replays the graph and launches
    the remainder; the result is that of direct launches, bit for bit."""
    ws = _mixed()
    a = batch_mod.Batch(ws)
    a.set_option(batch_mod.CUE_BOPT_MODE, mode)
    a.set_option(batch_mod.CUE_BOPT_ROWS, 8)
    a.run(2500)
    g = batch_mod.Batch(ws)
    g.set_option(batch_mod.CUE_BOPT_MODE, mode)
    g.set_option(batch_mod.CUE_BOPT_ROWS, 8)
    g.set_option(batch_mod.CUE_BOPT_GRAPH, 1)
    g.run(2500)
    a.check()
    g.check()
    assert g.get_option(batch_mod.CUE_BINFO_STEP) == 2500
    for i, w in enumerate(ws):
        _assert_same(a.snapshot(i), g.snapshot(i), w.name)
    assert a.cone_updates() == g.cone_updates()
    a.close()
    g.close()


@pytest.mark.parametrize("mode", [1, 2, 3])
@pytest.mark.parametrize("sample", ["c4-16", "mixed"])
def test_batched_step_matches_oracle(cue, batch_mod, sample, mode):
    """Every instance's batched step against the FP64 oracle's from the identical state: the
    batch runs 6 steps, each instance's state is copied out, then one more batched step must
    match one oracle step from that copy (field to FIELD_RTOL, cones as in the single-instance
    parity tests).  Samples: sixteen instances of the 512-instance workload, and the mixed set
    (nx % 4 = 0..3, stop radius, wall clamp, a rate map, no sources or cones)."""
    ws = W.config_c4(n_instances=16, nsteps=8) if sample == "c4-16" else _mixed()
    b = batch_mod.Batch(ws)
    b.set_option(batch_mod.CUE_BOPT_MODE, mode)
    after = 6
    b.run(after)
    b.check()
    before = [b.snapshot(i) for i in range(len(ws))]
    b.run(1)
    b.check()
    for i, w in enumerate(ws):
        C, pos, dirs, act = before[i]
        C1, pos1, dirs1, act1 = b.snapshot(i)
        want = oracle.field_step(grid_of(w), C.astype(np.float64), w.src_cell, w.src_emit, w.src_map)
        assert field_rel_err(C1, want) <= FIELD_RTOL, w.name
        if w.n_axons:
            compare_cones(w, C, after, pos, dirs, act, pos1, dirs1, act1)
    b.close()


def test_blocked_mode_on_clustered_and_crowded_instances(cue, batch_mod):
    """The blocked mode with every cone of an instance in one field tile (a 64 x 64 instance
    with 4,000 cones, a 900 x 700 instance whose 3,000 cones start in one corner), wall clamp
    and stop: bins beyond the 512 register slots, re-binning across tiles; bit for bit equal
    to each instance alone, over 2 x 8 + 3 steps."""
    rng = np.random.default_rng(90)
    a = W.make("crowd", 2, 64, 64, n_src=4, n_axons=4000, C0="smooth", seed=91)
    bw = W.make("corner", 2, 900, 700, n_src=12, n_axons=3000, C0="smooth", seed=92, wall_mode=1)
    bw.pos = rng.uniform(2.0, 40.0, (2, 3000)).astype(np.float32)
    ws = [a, bw]
    b = batch_mod.Batch(ws)
    b.set_option(batch_mod.CUE_BOPT_MODE, 3)
    b.set_option(batch_mod.CUE_BOPT_DEPTH, 8)
    b.run(19)
    b.check()
    for i, w in enumerate(ws):
        _assert_same(b.snapshot(i), _alone(cue, w, 19), w.name)
    b.close()


def _tile_boundary_instances():
    """Instances whose sides sit on either side of the blocked mode's tile-count steps at
    depths 2, 5 and 8 (halo H = K + 1 + ceil((K - 1) step_len / h): 3, 7 and 13 rows, 4, 8
    and 16 columns): one tile column up to 256 columns, one tile row up to 94 rows, then the
    first and last tiles ending at the walls; nx % 4 = 0..3, clamp and stop walls, a rate
    map, cones everywhere including the wall rows and columns."""
    rng = np.random.default_rng(95)
    sides = [(256, 94, 0), (257, 95, 1), (480, 164, 0), (481, 165, 1), (462, 150, 0), (463, 151, 1),
             (705, 235, 0), (99, 300, 1), (1030, 96, 0), (134, 143, 1)]
    out = []
    for k, (nx, ny, clamp) in enumerate(sides):
        w = W.make(f"edge{nx}x{ny}", 2, nx, ny, D=0.7 + 0.1 * k, lam=0.004, dt=0.2 / (0.7 + 0.1 * k), n_src=6 + k,
                   n_axons=300 + 40 * k, C0="smooth", seed=200 + k, wall_mode=clamp,
                   stop_radius=1.5 if k % 3 == 0 else 0.0, src_map="random" if k % 4 == 1 else False)
        # a quarter of the cones on the walls' nodes and the nodes next to them
        m = w.n_axons // 4
        side = rng.integers(0, 4, m)
        off = rng.uniform(0.0, 1.5, m)
        along_x = rng.uniform(0.0, nx - 1.0, m)
        along_y = rng.uniform(0.0, ny - 1.0, m)
        x = np.where(side == 0, off, np.where(side == 1, nx - 1.0 - off, along_x))
        y = np.where(side == 2, off, np.where(side == 3, ny - 1.0 - off, along_y))
        w.pos[0, :m] = x.astype(np.float32)
        w.pos[1, :m] = y.astype(np.float32)
        out.append(w)
    return out


@pytest.mark.parametrize("depth", [2, 5, 8])
def test_blocked_wall_aligned_tiles_at_count_boundaries(cue, batch_mod, depth):
    """Wall-aligned tiles of the blocked mode: instances whose sides straddle every step of
    the tile count (one tile, first and last tiles at the walls, middle tiles), bit for bit
    equal to each instance alone on the plain path over 3 launches plus a ragged one."""
    ws = _tile_boundary_instances()
    b = batch_mod.Batch(ws)
    b.set_option(batch_mod.CUE_BOPT_MODE, 3)
    b.set_option(batch_mod.CUE_BOPT_DEPTH, depth)
    nsteps = 3 * depth + 1
    b.run(nsteps)
    b.check()
    for i, w in enumerate(ws):
        _assert_same(b.snapshot(i), _alone(cue, w, nsteps), w.name)
    b.close()
