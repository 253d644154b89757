"""GPU (FP32, through the C ABI) vs FP64 oracle, one step from identical state.

Sizes span several thread blocks with ragged tails, the vectorised and the
any-size kernels, and the full benchmark grids (2D 2048^2 with 16,384 cones,
3D 256^3 with 65,536 cones).  Tolerances are in tests/parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1405_3331_gb300 import workloads as W
from parity import (FIELD_RTOL, POS_RTOL, ambiguous_cones, compare_cones, cone_of, field_rel_err, grid_of,
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


_compare_cones = compare_cones


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


def _on_walls(rng, dim, hi, n):
    """n uniform positions, each with one to dim coordinates moved onto a wall (0 or hi)."""
    pos = rng.uniform(0.0, 1.0, (dim, n)) * hi[:, None]
    for a in range(n):
        for ax in rng.choice(dim, int(rng.integers(1, dim + 1)), replace=False):
            pos[ax, a] = 0.0 if rng.integers(2) == 0 else hi[ax]
    return pos


@pytest.mark.parametrize("dim,wall_mode", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_cones_on_every_wall(cue, dim, wall_mode):
    """Cones exactly on the walls, edges and corners of every axis: the gradient is sampled in
    the clamped last cell (weight 1 on the far nodes) from wall nodes with ghost values, and the
    move takes the wall rule; the cone step alone and the coupled step against the oracle."""
    if dim == 2:
        w = W.make("walls2d", 2, 37, 29, n_src=3, n_axons=1, C0="smooth", seed=40, wall_mode=wall_mode)
    else:
        w = W.make("walls3d", 3, 21, 18, 15, dt=0.15, n_src=3, n_axons=1, C0="smooth", seed=41,
                   wall_mode=wall_mode)
    hi = (np.array([w.nx, w.ny, w.nz][:dim], np.float64) - 1) * w.h
    rng = np.random.default_rng(42 + dim)
    n = 3000
    w.pos = _on_walls(rng, dim, hi, n).astype(np.float32)
    d = rng.standard_normal((dim, n))
    w.dir = (d / np.linalg.norm(d, axis=0)).astype(np.float32)
    w.active = np.ones(n, np.uint8)
    C0 = w.field0()
    for run in (False, True):
        sim = _sim(cue, w, step=321)
        if run:
            sim.sim_run(1)
        else:
            sim.cone_step(1)
        sim.check()
        _, pos, dirs, act, _, _ = sim.snapshot()
        _compare_cones(w, C0, 321, w.pos, w.dir, w.active, pos, dirs, act)
        if wall_mode == 0:
            assert 0 < int((act == 0).sum()) < n          # some leave through a wall and stop
        else:
            assert act.all()
            assert ((pos >= 0) & (pos <= hi[:, None].astype(np.float32))).all()
        sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_stop_exactly_at_the_radius(cue, dim):
    """No cue and no noise (weights 1, 0, 0), axis-aligned moves of 0.5 onto or short of the stop
    radius 2 of a source: every quantity is exact in binary32, so the GPU must take the oracle's
    inclusive decision, ||p' - x||^2 <= r^2."""
    if dim == 2:
        w = W.make("radius2d", 2, 40, 30, n_src=1, n_axons=1, seed=43, stop_radius=2.0, w=(1.0, 0.0, 0.0))
        xs = np.array([12.0, 10.0])
        w.src_cell = np.array([12 + 40 * 10], np.int32)
    else:
        w = W.make("radius3d", 3, 20, 16, 12, dt=0.15, n_src=1, n_axons=1, seed=44, stop_radius=2.0,
                   w=(1.0, 0.0, 0.0))
        xs = np.array([6.0, 5.0, 4.0])
        w.src_cell = np.array([6 + 20 * (5 + 16 * 4)], np.int32)
    starts, heads, want_act = [], [], []
    for ax in range(dim):
        for sgn in (1.0, -1.0):
            e = np.zeros(dim)
            e[ax] = sgn
            for dist, stops in ((2.5, 0), (2.75, 1)):          # lands at 2.0 (stops) or 2.25
                starts.append(xs - dist * e)
                heads.append(e)
                want_act.append(stops)
    w.pos = np.array(starts, np.float32).T.copy()
    w.dir = np.array(heads, np.float32).T.copy()
    w.active = np.ones(len(starts), np.uint8)
    for run in (False, True):
        sim = _sim(cue, w, step=5)
        if run:
            sim.sim_run(1)
        else:
            sim.cone_step(1)
        sim.check()
        _, pos, dirs, act, _, _ = sim.snapshot()
        np.testing.assert_array_equal(pos, w.pos + 0.5 * w.dir)
        np.testing.assert_array_equal(act, want_act)
        _, _, ract = oracle.cone_step(grid_of(w), cone_of(w), w.field0().astype(np.float64), 5, w.pos,
                                      w.dir, w.active, w.src_cell)
        np.testing.assert_array_equal(act, ract)
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


@pytest.mark.parametrize("layout", ["crowded", "stop"])
def test_one_launch_3d_cones_over_many_steps(cue, layout):
    """The one-launch 3D step over 150 steps in two calls with crowded cones ('crowded':
    3,000 of 3,500 cones in one z plane of one column tile, gathering the same nodes) and
    with a source-stop radius ('stop': cones drop out as they stop).  Bit for bit equal to
    the separate cone and field launches."""
    if layout == "crowded":
        w = W.make("3d-crowd", 3, 64, 48, 40, dt=0.15, n_src=6, n_axons=3500, C0="smooth", seed=61)
        rng = np.random.default_rng(61)
        w.pos[:2, :3000] = rng.uniform(4.0, 12.0, (2, 3000)).astype(np.float32)
        w.pos[2, :3000] = rng.uniform(5.1, 5.9, 3000).astype(np.float32)   # one z plane: one box
    else:
        w = W.make("3d-stop", 3, 64, 48, 40, dt=0.15, n_src=12, n_axons=2000, C0="smooth", seed=62,
                   stop_radius=2.5)
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    b = cue.Simulation(w, path=cue.CUE_PATH_PLAIN, field_offset=1)
    for n in (70, 80):
        a.sim_run(n)
        b.sim_run(n)
    a.check()
    b.check()
    sa, sb = a.snapshot(), b.snapshot()
    for x, y in zip(sa[:4], sb[:4]):
        np.testing.assert_array_equal(x, y)
    assert a.cone_updates() == b.cone_updates()
    if layout == "stop":
        assert 0 < int(sa[3].sum()) < w.n_axons            # some cones stopped, some still move
    a.close()
    b.close()


def _max_case(dim):
    """The largest grids the library accepts (fewer than 2^31 nodes): 65536 x 32767 and
    1288 x 1288 x 1294, nx % 4 == 0 so the aligned kernels run."""
    if dim == 2:
        return 65536, 32767, 1
    return 1288, 1288, 1294


def _padded(field_t, origin, size):
    """Input values of a window grown by one node on every side, NaN outside the grid."""
    import torch
    dim = field_t.dim()
    ext = list(reversed(field_t.shape))                           # x, y(, z)
    lo = [max(o - 1, 0) for o in origin]
    hi = [min(o + s + 1, e) for o, s, e in zip(origin, size, ext)]
    sl = tuple(slice(l, h) for l, h in zip(reversed(lo), reversed(hi)))
    block = field_t[sl].to(torch.float64).cpu().numpy()
    Wp = np.full(tuple(s + 2 for s in reversed(size)), np.nan)
    off = tuple(slice(l - (o - 1), l - (o - 1) + n) for l, o, n in zip(reversed(lo), reversed(origin), block.shape))
    Wp[off] = block
    return Wp


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("offset", [0, 1])
def test_maximum_grid_one_step_on_sampled_windows(cue, dim, offset):
    """One coupled step on the largest accepted grid, through the aligned path (fused in 2D,
    the TMA step kernel in 3D) and through the any-size kernels (a one-float offset), against
    the oracle's windowed step on windows at the first and last nodes, along the walls, in
    the middle and around sources at the first node, the last node and high linear indices;
    the cones near the far corner move by exactly one step length."""
    import torch
    nx, ny, nz = _max_case(dim)
    n = nx * ny * nz
    assert n < 2 ** 31 - 1
    free, _ = torch.cuda.mem_get_info()
    if free < 2.5 * 2 * 4 * n:
        pytest.skip("not enough device memory for two fields of 2^31 nodes")
    w = W.make(f"max-{dim}d", dim, nx, ny, nz, dt=0.15 if dim == 3 else 0.2, n_src=4, n_axons=256,
               emit=(0.5, 2.0), seed=30 + dim)
    ext = (nx, ny, nz)[:dim]
    w.src_cell = np.array([0, n - 1, n - 1 - 3 * nx, n // 2 + 5], np.int32)
    rng = np.random.default_rng(31)
    w.pos = (np.array(ext, np.float32)[:, None] - 3.0
             - rng.uniform(0.0, 6.0, (dim, w.n_axons)).astype(np.float32) * (np.array(ext)[:, None] > 8))
    w.pos = np.clip(w.pos, 0.5, None).astype(np.float32)
    shape = w.shape
    w.field0 = lambda: torch.zeros((), dtype=torch.float32, device="cuda:0").expand(shape)
    path = cue.CUE_PATH_PLAIN if offset else cue.CUE_PATH_AUTO
    sim = cue.Simulation(w, path=path, field_offset=offset)
    # a separable field: random along each axis, summed (no temporaries of the grid's size)
    g = torch.Generator(device="cuda:0").manual_seed(32 + dim)
    axes = [torch.rand(s, generator=g, device="cuda:0") for s in reversed(ext)]    # z?, y, x
    f0 = sim.fields[0]
    if dim == 2:
        torch.add(axes[0][:, None], axes[1][None, :], out=f0)
    else:
        torch.add((axes[0][:, None] + axes[1][None, :])[:, :, None], axes[2][None, None, :], out=f0)
    torch.cuda.synchronize()
    if dim == 2:
        windows = [((0, 0), (8, 6)), ((nx - 8, ny - 6), (8, 6)), ((nx // 2, 0), (8, 3)), ((0, ny // 2), (4, 6)),
                   ((nx // 2 - 4, ny // 2 - 3), (12, 8)), ((nx - 12, ny - 8), (12, 8))]
    else:
        windows = [((0, 0, 0), (8, 4, 3)), ((nx - 8, ny - 4, nz - 3), (8, 4, 3)), ((nx // 2, 0, nz // 2), (8, 3, 3)),
                   ((0, ny // 2, nz - 2), (4, 5, 2)), ((nx // 2 - 4, ny // 2 - 2, nz // 2 - 1), (12, 6, 4))]
    src_xyz = [((c % nx), (c // nx) % ny, c // (nx * ny)) for c in w.src_cell.astype(np.int64)]
    for c in src_xyz[2:]:                               # windows around the sources at high indices
        o = [max(0, min(c[a] - 2, ext[a] - 5)) for a in range(dim)]
        windows.append((tuple(o), (5,) * dim))
    inputs = [_padded(f0, o, s) for o, s in windows]
    pos0, dir0, act0 = sim.pos.cpu().numpy(), sim.dir.cpu().numpy(), sim.active.cpu().numpy()
    sim.sim_run(1)
    sim.check()
    out = sim.field()
    grid = grid_of(w)
    emit = w.src_emit.astype(np.float64)
    for (o, s), Wp in zip(windows, inputs):
        want = oracle.field_window(grid, Wp, o, w.src_cell.astype(np.int64), emit)
        sl = tuple(slice(a, a + b) for a, b in zip(reversed(o), reversed(s)))
        got = out[sl].cpu().numpy()
        assert field_rel_err(got, want) <= FIELD_RTOL, (o, s)
    pos1, dir1, act1 = sim.pos.cpu().numpy(), sim.dir.cpu().numpy(), sim.active.cpu().numpy()
    moved = act0.astype(bool) & act1.astype(bool)
    assert moved.sum() > 0.9 * w.n_axons
    step = np.linalg.norm(pos1.astype(np.float64) - pos0, axis=0)
    np.testing.assert_allclose(step[moved], w.step_len, atol=0.02)      # float32 ulp at x ~ 65536 is 0.004
    np.testing.assert_allclose(np.linalg.norm(dir1[:, moved].astype(np.float64), axis=0), 1.0, atol=1e-5)
    assert sim.last_path() == (cue.CUE_PATH_FUSED if (dim == 2 and not offset) else cue.CUE_PATH_PLAIN)
    sim.close()
    del sim, f0, out
    torch.cuda.empty_cache()
