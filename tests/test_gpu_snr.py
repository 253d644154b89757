"""The SNR turn rule (Sec. 3.5, Eq. 5) on the GPU against the FP64 oracle.

A decision is the sign of SNR + z; FP32 and FP64 take it alike except when
SNR + z is within rounding of 0, or C(p) within rounding of a window edge, or
the trial position within rounding of a wall or of a source's stop radius:
those cones are excluded (and counted, at most 1%), every other cone must
match position, direction and stop flag to the per-step bar.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1405_3331_gb300 import workloads as W
from parity import POS_RTOL, grid_of, pos_rel_err

pytestmark = pytest.mark.gpu

SNR = dict(gain=8.0, width=2.0, kd=1.5, c_min=0.05, c_max=50.0, turn=math.pi / 30)


@pytest.fixture(scope="module")
def cue():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import cue as binding
    return binding


def _cone(w, snr=SNR):
    return oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps, w.wall_mode, w.seed,
                       steer=1, snr_gain=snr["gain"], snr_width=snr["width"], snr_kd=snr["kd"],
                       snr_cmin=snr["c_min"], snr_cmax=snr["c_max"], snr_turn=snr["turn"])


def _case(name):
    if name == "stop-256x192":
        return W.make(name, 2, 256, 192, n_src=6, n_axons=4000, C0="smooth", seed=80, stop_radius=2.0)
    if name == "clamp-300x212":
        return W.make(name, 2, 300, 212, n_src=9, n_axons=3000, C0="smooth", seed=81, wall_mode=1)
    if name == "odd-131x77":
        return W.make(name, 2, 131, 77, n_src=3, n_axons=500, C0="random", seed=82)
    raise KeyError(name)


def _ambiguous(w, c, C, step, pos, d, act, margin=1e-4):
    g = grid_of(w)
    n = act.shape[0]
    p = np.asarray(pos, np.float64)
    Cp = oracle.value_at(g, C, p.T)
    grads = oracle.gradient_at(g, C, p.T)[:, :2]
    z = oracle.noise(w.seed, np.arange(n), step, 2)[:, 0]
    amb = np.zeros(n, bool)
    for a in range(n):
        s = oracle.snr(c, Cp[a], grads[a], d[:, a])
        amb[a] = abs(s + z[a]) <= margin * (1.0 + abs(s))
    amb |= np.abs(Cp - c.snr_cmin) <= margin * np.maximum(np.abs(Cp), 1.0)
    amb |= np.abs(Cp - c.snr_cmax) <= margin * np.maximum(np.abs(Cp), 1.0)
    free = oracle.Cone(**{**c.__dict__, "stop_radius": 0.0, "wall_mode": 1})
    _, d_trial, _ = oracle.cone_step(g, free, C, step, p, d, np.ones(n, np.uint8))
    trial = p + w.step_len * d_trial
    hi = np.array([(w.nx - 1) * w.h, (w.ny - 1) * w.h])[:, None]
    amb |= np.minimum(np.abs(trial), np.abs(trial - hi)).min(axis=0) <= margin * np.maximum(np.linalg.norm(p, axis=0), 1.0)
    if w.stop_radius > 0 and w.n_src > 0:
        cells = w.src_cell.astype(np.int64)
        xs = np.stack([(cells % w.nx) * w.h, (cells // w.nx) * w.h])
        d2 = ((trial[:, :, None] - xs[:, None, :]) ** 2).sum(0)
        amb |= (np.abs(d2 - w.stop_radius ** 2) <= margin * 10 * w.stop_radius ** 2).any(axis=1)
    return amb & act.astype(bool)


@pytest.mark.parametrize("name", ["stop-256x192", "clamp-300x212", "odd-131x77"])
@pytest.mark.parametrize("step", [0, 37])
def test_snr_cone_step_matches_oracle(cue, name, step):
    w = _case(name)
    sim = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    sim.set_steering(SNR)
    sim.load(step=step)
    sim.cone_step(1)
    sim.check()
    _, pos, dirs, act, _, _ = sim.snapshot()
    sim.close()
    c = _cone(w)
    C = w.field0().astype(np.float64)
    want_p, want_d, want_a = oracle.cone_step(grid_of(w), c, C, step, w.pos, w.dir, w.active, w.src_cell)
    keep = ~_ambiguous(w, c, C, step, w.pos.astype(np.float64), w.dir.astype(np.float64), w.active)
    assert (~keep).sum() <= max(2, 0.01 * w.n_axons)
    np.testing.assert_array_equal(act[keep], want_a[keep])
    assert pos_rel_err(pos[:, keep], want_p[:, keep]).max() <= POS_RTOL
    assert np.abs(dirs[:, keep] - want_d[:, keep]).max() <= 1e-5
    turned = np.abs(dirs[0] * w.dir[1] - dirs[1] * w.dir[0]) > 1e-3
    assert turned.mean() > 0.3                                 # the rule is at work


@pytest.mark.parametrize("name", ["stop-256x192", "clamp-300x212"])
def test_snr_persistent_equals_plain_bitwise(cue, name):
    w = _case(name)
    out = []
    for path in (cue.CUE_PATH_PLAIN, cue.CUE_PATH_PERSIST):
        sim = cue.Simulation(w, path=path)
        sim.set_steering(SNR)
        sim.sim_run(30)
        sim.check()
        out.append(sim.snapshot())
        assert sim.last_path() == path
        sim.close()
    for x, y in zip(out[0][:4], out[1][:4]):
        assert np.array_equal(x, y)


def test_flat_field_turns_are_a_fair_coin(cue):
    w = W.make("flat", 2, 128, 128, n_src=0, n_axons=40000, seed=83)
    w.C0 = np.full(w.shape, 2.0, np.float32)
    sim = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    sim.set_steering(SNR)
    sim.cone_step(1)
    sim.check()
    _, pos, dirs, act, _, _ = sim.snapshot()
    sim.close()
    cross = w.dir[0].astype(np.float64) * dirs[1] - w.dir[1].astype(np.float64) * dirs[0]
    ok = act.astype(bool)
    right = np.mean(cross[ok] < 0)
    assert abs(right - 0.5) < 4 * math.sqrt(0.25 / ok.sum())
    np.testing.assert_allclose(np.abs(cross[ok]), math.sin(math.pi / 30), atol=2e-6)


def test_steering_switch_and_refusals(cue):
    w = _case("odd-131x77")
    ref = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    ref.sim_run(5)
    a = cue.Simulation(w, path=cue.CUE_PATH_PLAIN)
    a.set_steering(SNR)
    a.set_steering(None)                                        # back to vector addition
    a.sim_run(5)
    for x, y in zip(ref.snapshot()[:4], a.snapshot()[:4]):
        assert np.array_equal(x, y)
    with pytest.raises(cue.CueError):
        a.set_steering(dict(SNR, kd=0.0))
    with pytest.raises(cue.CueError):
        a.set_steering(dict(SNR, c_min=3.0, c_max=1.0))
    ref.close()
    a.close()
    w3 = W.make("snr3d", 3, 16, 16, 16, dt=0.15, n_src=2, n_axons=10, seed=84)
    s3 = cue.Simulation(w3)
    with pytest.raises(cue.CueError):
        s3.set_steering(SNR)
    s3.close()
    w2 = W.make("snrfused", 2, 256, 256, n_src=4, n_axons=100, C0="smooth", seed=85)
    s2 = cue.Simulation(w2)
    s2.set_steering(SNR)
    with pytest.raises(cue.CueError):
        s2.set_option(cue.CUE_OPT_PATH, cue.CUE_PATH_FUSED)
    s2.sim_run(3)
    s2.check()
    assert s2.last_path() != cue.CUE_PATH_FUSED
    s2.close()
    wa = W.config_c5(n=64, n_src=2, n_axons=16, nsteps=10)
    sa = cue.Simulation(wa)
    sa.set_steering(SNR)
    with pytest.raises(cue.CueError):
        sa.adjoint(wa.targets, 10, 4)
    sa.close()
