"""The shared-memory resident 2D path (one block holds the grid in shared memory
and the cones in registers for a whole call).

Per node and per cone it computes the plain path's arithmetic in the same
order, so the two must agree bit for bit (source cells are distinct in these
workloads), both field buffers included; calls must continue one another; AUTO
must take it exactly where it applies.
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
        return W.make(name, 2, 128, 128, lam=0.01, n_src=4, n_axons=64, C0="smooth", seed=70)
    if name == "4x2":
        return W.make(name, 2, 4, 2, n_src=1, n_axons=3, C0="random", seed=71)
    if name == "8x8":
        return W.make(name, 2, 8, 8, n_src=2, n_axons=16, C0="random", seed=72)
    if name == "100x37-stop":
        return W.make(name, 2, 100, 37, n_src=9, n_axons=200, C0="smooth", seed=73, stop_radius=2.0)
    if name == "map-96x64-clamp":
        return W.make(name, 2, 96, 64, n_src=6, n_axons=128, C0="smooth", seed=74, src_map="random",
                      wall_mode=1)
    if name == "160x160-256cones":
        return W.make(name, 2, 160, 160, n_src=40, n_axons=256, C0="smooth", seed=75, stop_radius=1.5)
    if name == "field-only":
        return W.make(name, 2, 64, 48, n_src=3, n_axons=0, C0="smooth", seed=76)
    if name == "no-sources":
        return W.make(name, 2, 64, 48, n_src=0, n_axons=40, C0="smooth", seed=77)
    if name == "4x2000-tall":                       # bands of 65 rows: the row bitmap is read in pieces
        return W.make(name, 2, 4, 2000, n_src=30, n_axons=20, C0="smooth", seed=82, stop_radius=1.0)
    raise KeyError(name)


CASES = ["c1-128", "4x2", "8x8", "100x37-stop", "map-96x64-clamp", "160x160-256cones", "field-only",
         "no-sources", "4x2000-tall"]


def _run(cue, w, path, calls, snr=None):
    sim = cue.Simulation(w, path=path)
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


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("nsteps", [1, 2, 37])
def test_resident_equals_plain_bitwise(cue, name, nsteps):
    w = _case(name)
    a, pa = _run(cue, w, cue.CUE_PATH_PLAIN, [nsteps])
    b, pb = _run(cue, w, cue.CUE_PATH_RESIDENT, [nsteps])
    assert pa == cue.CUE_PATH_PLAIN and pb == cue.CUE_PATH_RESIDENT
    _assert_same(a, b)


@pytest.mark.parametrize("name", ["c1-128", "100x37-stop"])
def test_resident_equals_persistent_with_the_snr_rule(cue, name):
    w = _case(name)
    a, pa = _run(cue, w, cue.CUE_PATH_PERSIST, [30], snr=SNR)
    b, pb = _run(cue, w, cue.CUE_PATH_RESIDENT, [30], snr=SNR)
    assert pa == cue.CUE_PATH_PERSIST and pb == cue.CUE_PATH_RESIDENT
    _assert_same(a, b)


def test_calls_continue_one_another(cue):
    """Step counter, Philox step and buffer parity carry over between calls."""
    w = _case("100x37-stop")
    ref, _ = _run(cue, w, cue.CUE_PATH_PLAIN, [12])
    got, used = _run(cue, w, cue.CUE_PATH_RESIDENT, [5, 0, 1, 6])
    assert used == cue.CUE_PATH_RESIDENT
    _assert_same(ref, got)


def test_auto_takes_the_resident_path_where_it_applies(cue):
    """Grids below the cluster path's 4,096 nodes, or with fewer rows than its bands need."""
    for w in (W.make("short", 2, 128, 12, n_src=3, n_axons=40, C0="smooth", seed=83),
              W.make("64x48", 2, 64, 48, n_src=3, n_axons=40, C0="smooth", seed=84, src_map="random"),
              W.make("32x32", 2, 32, 32, n_src=2, n_axons=16, C0="smooth", seed=85)):
        sim = cue.Simulation(w)
        sim.sim_run(3)
        sim.check()
        assert sim.last_path() == cue.CUE_PATH_RESIDENT, w.name
        sim.close()
    # too many cones for the cone warps, or both buffers beyond one block's shared memory: the
    # resident path is refused (AUTO takes the cluster path there)
    for w in (W.make("cones", 2, 128, 128, n_src=4, n_axons=257, seed=78),
              W.make("big", 2, 256, 192, n_src=4, n_axons=64, seed=79)):
        sim = cue.Simulation(w)
        sim.sim_run(2)
        sim.check()
        assert sim.last_path() == cue.CUE_PATH_CLUSTER, w.name
        with pytest.raises(cue.CueError) as e:
            sim.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_RESIDENT)
        assert e.value.code == cue.CUE_ERR_ARG
        sim.close()


def test_one_resident_step_matches_oracle(cue):
    w = _case("map-96x64-clamp")
    sim = cue.Simulation(w, path=cue.CUE_PATH_RESIDENT)
    sim.load(step=91)
    sim.sim_run(1)
    sim.check()
    assert sim.last_path() == cue.CUE_PATH_RESIDENT
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
    w = W.make("bounds", 2, 64, 64, n_src=3, n_axons=8, C0="smooth", seed=80)
    w.src_cell = np.array([5, 64 * 64 + 7, -3], np.int32)
    sim = cue.Simulation(w, path=cue.CUE_PATH_RESIDENT)
    sim.status()                                        # the handle's own source pass already saw them
    sim.sim_run(1)
    assert sim.status() == cue.CUE_ERR_BOUNDS
    assert sim.last_path() == cue.CUE_PATH_RESIDENT
    got = sim.field().cpu().numpy()
    want = oracle.field_step(grid_of(w), w.field0().astype(np.float64), [5], w.src_emit[:1])
    assert field_rel_err(got, want) <= FIELD_RTOL
    sim.close()


def test_nonfinite_is_reported(cue):
    w = W.make("nan", 2, 64, 64, n_src=1, n_axons=4, C0="smooth", seed=81)
    w.C0 = w.field0()
    w.C0[10, 10] = np.nan
    sim = cue.Simulation(w, path=cue.CUE_PATH_RESIDENT)
    sim.sim_run(2)
    assert sim.status() == cue.CUE_ERR_NONFINITE
    sim.close()
