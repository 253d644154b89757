"""The thread-block-cluster 2D path (a cluster of 8 or 16 CTAs holds the grid
in distributed shared memory, one band of rows each, for a whole call).

Per node and per cone it computes the plain path's arithmetic in the same
order, so the two must agree bit for bit (source cells are distinct in these
workloads), both field buffers included, at either cluster size; band edge
rows reach the neighbouring CTA's halo through distributed shared memory
stores, and cones whose patch crosses a band edge read the neighbour's
shared memory; calls must continue one another; AUTO must take it exactly
where it applies.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1405_3331_gb300 import workloads as W
from parity import FIELD_RTOL, POS_RTOL, ambiguous_cones, cone_of, field_rel_err, grid_of, pos_rel_err

pytestmark = pytest.mark.gpu

SNR = dict(gain=8.0, width=2.0, kd=1.5, c_min=0.05, c_max=50.0, turn=math.pi / 30)


@pytest.fixture(scope="module")
def cue():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


def _case(name):
    if name == "c1-128":
        return W.make(name, 2, 128, 128, lam=0.01, n_src=4, n_axons=64, C0="smooth", seed=170)
    if name == "16x16":                             # bands of 2 rows: every patch spans bands
        return W.make(name, 2, 16, 16, n_src=2, n_axons=16, C0="random", seed=171)
    if name == "100x37-stop":                       # bands of 5 rows, the last one 2
        return W.make(name, 2, 100, 37, n_src=9, n_axons=200, C0="smooth", seed=173, stop_radius=2.0)
    if name == "map-96x64-clamp":
        return W.make(name, 2, 96, 64, n_src=6, n_axons=128, C0="smooth", seed=174, src_map="random",
                      wall_mode=1)
    if name == "256x192-2000cones":                 # beyond the single block's shared memory
        return W.make(name, 2, 256, 192, n_src=40, n_axons=2000, C0="smooth", seed=175, stop_radius=1.5)
    if name == "field-only":
        return W.make(name, 2, 64, 48, n_src=3, n_axons=0, C0="smooth", seed=176)
    if name == "no-sources":
        return W.make(name, 2, 64, 48, n_src=0, n_axons=40, C0="smooth", seed=177)
    if name == "4x2000-tall":
        return W.make(name, 2, 4, 2000, n_src=30, n_axons=20, C0="smooth", seed=182, stop_radius=1.0)
    raise KeyError(name)


CASES = ["c1-128", "16x16", "100x37-stop", "map-96x64-clamp", "256x192-2000cones", "field-only", "no-sources",
         "4x2000-tall"]


def _run(cue, w, path, calls, snr=None, ctas=0):
    sim = cue.Simulation(w, path=path)
    if ctas:
        try:
            sim.set_option(cue.CUE_OPT_CLUSTER_CTAS, ctas)
        except cue.CueError:
            sim.close()
            pytest.skip(f"no {ctas}-CTA cluster of this size can be scheduled on this device")
    if snr:
        sim.set_steering(snr)
    for k in calls:
        sim.sim_run(k)
    sim.check()
    out = sim.snapshot() + (sim.fields[0].cpu().numpy(), sim.fields[1].cpu().numpy(), sim.cone_updates())
    used = sim.last_path()
    sim.close()
    return out, used


def _assert_same(sa, sb):
    names = ("field", "pos", "dir", "active", "field step", "cone step", "buffer 0", "buffer 1", "cone updates")
    for x, y, what in zip(sa, sb, names):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y), f"{what} differs: max {np.abs(x.astype(float) - y.astype(float)).max()}"
        else:
            assert x == y, (what, x, y)


@pytest.mark.parametrize("ctas", [8, 16])
@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("nsteps", [1, 2, 37])
def test_cluster_equals_plain_bitwise(cue, name, nsteps, ctas):
    w = _case(name)
    if w.ny < 2 * ctas:
        pytest.skip("a band per CTA needs two rows")
    a, pa = _run(cue, w, cue.CUE_PATH_PLAIN, [nsteps])
    b, pb = _run(cue, w, cue.CUE_PATH_CLUSTER, [nsteps], ctas=ctas)
    assert pa == cue.CUE_PATH_PLAIN and pb == cue.CUE_PATH_CLUSTER
    _assert_same(a, b)


@pytest.mark.parametrize("ctas", [8, 16])
@pytest.mark.parametrize("name", ["c1-128", "100x37-stop"])
def test_cluster_equals_resident_with_the_snr_rule(cue, name, ctas):
    w = _case(name)
    a, pa = _run(cue, w, cue.CUE_PATH_RESIDENT, [30], snr=SNR)
    b, pb = _run(cue, w, cue.CUE_PATH_CLUSTER, [30], snr=SNR, ctas=ctas)
    assert pa == cue.CUE_PATH_RESIDENT and pb == cue.CUE_PATH_CLUSTER
    _assert_same(a, b)


@pytest.mark.parametrize("ctas", [8, 16])
def test_cluster_whole_c1_run_equals_resident(cue, ctas):
    """The 128^2 workload's 500 steps in one call: cluster and resident paths agree bit for
    bit over the whole run (the cones wander across every band edge)."""
    w = W.config_c1()
    a, _ = _run(cue, w, cue.CUE_PATH_RESIDENT, [500])
    b, pb = _run(cue, w, cue.CUE_PATH_CLUSTER, [500], ctas=ctas)
    assert pb == cue.CUE_PATH_CLUSTER
    _assert_same(a, b)


def test_cluster_size_option(cue):
    """CUE_OPT_CLUSTER_CTAS takes 0, 8 or 16; CUE_INFO_GRID reports the CTAs of the last
    cluster launch; a size the grid cannot take (16 CTAs need 32 rows) is refused while the
    cluster path is selected, and the old size kept."""
    w = _case("c1-128")
    sim = cue.Simulation(w, path=cue.CUE_PATH_CLUSTER)
    assert sim.get_option(cue.CUE_OPT_CLUSTER_CTAS) == 0
    for bad in (1, 4, 12, 32, -8):
        with pytest.raises(cue.CueError):
            sim.set_option(cue.CUE_OPT_CLUSTER_CTAS, bad)
    sim.set_option(cue.CUE_OPT_CLUSTER_CTAS, 8)
    sim.sim_run(2)
    sim.check()
    assert sim.get_option(cue.CUE_INFO_GRID) == 8
    sim.close()
    short = W.make("rows-24", 2, 64, 24, n_src=2, n_axons=8, C0="smooth", seed=184)
    sim = cue.Simulation(short, path=cue.CUE_PATH_CLUSTER)
    with pytest.raises(cue.CueError):
        sim.set_option(cue.CUE_OPT_CLUSTER_CTAS, 16)
    assert sim.get_option(cue.CUE_OPT_CLUSTER_CTAS) == 0
    sim.sim_run(1)
    sim.check()
    assert sim.get_option(cue.CUE_INFO_GRID) == 8
    sim.close()


def test_cones_beyond_one_warp_per_band(cue):
    """4,000 cones on 8 CTAs (16 cone warps each, the most a CTA takes) and 8,000 on 16:
    every cone lane of every CTA busy, bit for bit equal to the plain path."""
    for ctas, n in ((8, 4000), (16, 8000)):
        w = W.make(f"cones-{n}", 2, 128, 160, n_src=12, n_axons=n, C0="smooth", seed=185 + ctas, stop_radius=1.0)
        a, _ = _run(cue, w, cue.CUE_PATH_PLAIN, [9])
        b, pb = _run(cue, w, cue.CUE_PATH_CLUSTER, [9], ctas=ctas)
        assert pb == cue.CUE_PATH_CLUSTER
        _assert_same(a, b)


def test_calls_continue_one_another(cue):
    """Step counter, Philox step and buffer parity carry over between calls."""
    w = _case("100x37-stop")
    ref, _ = _run(cue, w, cue.CUE_PATH_PLAIN, [12])
    got, used = _run(cue, w, cue.CUE_PATH_CLUSTER, [5, 0, 1, 6])
    assert used == cue.CUE_PATH_CLUSTER
    _assert_same(ref, got)


def test_auto_takes_the_cluster_path_where_it_applies(cue):
    """At least 4,096 nodes, at most 128 cones and 16,384 nodes per CTA."""
    for w in (_case("c1-128"), _case("map-96x64-clamp"), _case("256x192-2000cones"),
              W.make("map-300x212", 2, 300, 212, n_src=9, n_axons=500, C0="smooth", seed=183, src_map="random",
                     wall_mode=1)):
        sim = cue.Simulation(w)
        sim.sim_run(3)
        sim.check()
        assert sim.last_path() == cue.CUE_PATH_CLUSTER, w.name
        sim.close()
    # below 4,096 nodes or 16 rows: the single block; more cones per CTA: the persistent
    # kernel, though the cluster path can still be selected where it fits
    for w, want, selectable in (
            (W.make("short", 2, 64, 12, n_src=2, n_axons=8, seed=178), cue.CUE_PATH_RESIDENT, False),
            (W.make("64x48", 2, 64, 48, n_src=2, n_axons=8, seed=186), cue.CUE_PATH_RESIDENT, True),
            (W.make("64x1000", 2, 64, 1000, n_src=20, n_axons=3000, seed=187), cue.CUE_PATH_PERSIST, True),
            (W.make("cones", 2, 128, 128, n_src=4, n_axons=8193, seed=179), cue.CUE_PATH_PERSIST, False)):
        sim = cue.Simulation(w)
        sim.sim_run(2)
        sim.check()
        assert sim.last_path() == want, w.name
        if selectable:
            sim.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_CLUSTER)
            sim.sim_run(1)
            sim.check()
            assert sim.last_path() == cue.CUE_PATH_CLUSTER, w.name
        else:
            with pytest.raises(cue.CueError) as e:
                sim.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_CLUSTER)
            assert e.value.code == cue.CUE_ERR_ARG
        sim.close()


def test_one_cluster_step_matches_oracle(cue):
    w = _case("map-96x64-clamp")
    sim = cue.Simulation(w, path=cue.CUE_PATH_CLUSTER)
    sim.load(step=91)
    sim.sim_run(1)
    sim.check()
    assert sim.last_path() == cue.CUE_PATH_CLUSTER
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


def test_out_of_range_sources_are_reported_and_skipped(cue):
    w = W.make("bounds", 2, 64, 64, n_src=3, n_axons=8, C0="smooth", seed=180)
    w.src_cell = np.array([5, 64 * 64 + 7, -3], np.int32)
    sim = cue.Simulation(w, path=cue.CUE_PATH_CLUSTER)
    sim.status()                                        # the handle's own source pass already saw them
    sim.sim_run(1)
    assert sim.status() == cue.CUE_ERR_BOUNDS
    assert sim.last_path() == cue.CUE_PATH_CLUSTER
    got = sim.field().cpu().numpy()
    want = oracle.field_step(grid_of(w), w.field0().astype(np.float64), [5], w.src_emit[:1])
    assert field_rel_err(got, want) <= FIELD_RTOL
    sim.close()


def test_nonfinite_is_reported(cue):
    w = W.make("nan", 2, 64, 64, n_src=1, n_axons=4, C0="smooth", seed=181)
    w.C0 = w.field0()
    w.C0[10, 10] = np.nan
    sim = cue.Simulation(w, path=cue.CUE_PATH_CLUSTER)
    sim.sim_run(2)
    assert sim.status() == cue.CUE_ERR_NONFINITE
    sim.close()


def test_cluster_at_its_largest_grid(cue):
    """1024 x 400 on 16 CTAs: bands of 25 rows, both buffers and the halo rows take
    (25 + 2) x 1024 x 8 B = 221 KB of a CTA's 227 KB; bit for bit equal to the plain path,
    every cone lane busy across band edges.  Sixteen more rows (bands of 26) no longer fit
    in one block's shared memory, so the cluster path is refused there."""
    w = W.make("1024x400", 2, 1024, 400, n_src=40, n_axons=2000, C0="smooth", seed=188, stop_radius=1.0)
    a, _ = _run(cue, w, cue.CUE_PATH_PLAIN, [3])
    b, pb = _run(cue, w, cue.CUE_PATH_CLUSTER, [3], ctas=16)
    assert pb == cue.CUE_PATH_CLUSTER
    _assert_same(a, b)
    big = W.make("1024x416", 2, 1024, 416, n_src=4, n_axons=64, C0="smooth", seed=189)
    sim = cue.Simulation(big)
    with pytest.raises(cue.CueError) as e:
        sim.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_CLUSTER)
    assert e.value.code == cue.CUE_ERR_ARG
    sim.close()
