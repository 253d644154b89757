"""Pins of the oracle's SNR turn rule (Sec. 3.5, Eq. 5), CPU only.

The rule: inside the detectable concentration window the cone turns by the
turn angle (pi/30 in the paper) to the right when a draw from N(SNR, 1) is
positive, else to the left; outside the window it keeps its direction.  The
pins check what the rule fixes without re-deriving Eq. 5: the closed-form
heading sequence when the SNR dwarfs the unit-variance draw, the flat-field
case (SNR = 0, a fair coin), the mirror symmetry of the decision, the window,
and the decision law P(right) = Phi(SNR) over many independent cones.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import Cone, Grid

TURN = math.pi / 30


def _ramp(nx=200, ny=200, c0=1.0, slope=0.01):
    """C = c0 + slope * x: the interior node gradients are exactly (slope, 0)."""
    x = np.arange(nx, dtype=np.float64)
    return np.tile(c0 + slope * x, (ny, 1))


def _snr_cone(**kw):
    d = dict(step_len=0.5, wall_mode=1, seed=99, steer=1, snr_gain=1.0, snr_width=1.0, snr_kd=1.0,
             snr_cmin=0.0, snr_cmax=1e30)
    d.update(kw)
    return Cone(**d)


def test_huge_snr_turns_by_the_closed_form_sequence():
    """Gradient along +x (theta_NGF = 0), heading theta0 = pi/2 + 0.05: with the SNR far above
    any unit-normal draw the cone turns right (clockwise) while sin(theta) > 0, i.e. 16 times,
    then alternates around the gradient direction; each step advances along the new heading."""
    g = Grid(2, 200, 200, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = _ramp()
    c = _snr_cone(snr_gain=1e6)
    th0 = math.pi / 2 + 0.05
    p0 = np.array([[60.0], [100.0]])
    d0 = np.array([[math.cos(th0)], [math.sin(th0)]])
    T = 24
    th, thetas = th0, []
    for k in range(T):
        th = th - TURN if math.sin(th) > 0 else th + TURN
        thetas.append(th)
    assert sum(1 for a, b in zip([th0] + thetas, thetas) if b < a) >= 16
    pos, dirs = p0.copy(), d0.copy()
    want_p = p0[:, 0].copy()
    for k in range(T):
        _, pos, dirs, act = oracle.run(g, c, C, k, 1, (), (), None, pos, dirs, np.ones(1, np.uint8))
        want_p = want_p + 0.5 * np.array([math.cos(thetas[k]), math.sin(thetas[k])])
        np.testing.assert_allclose(dirs[:, 0], [math.cos(thetas[k]), math.sin(thetas[k])], atol=1e-12)
        np.testing.assert_allclose(pos[:, 0], want_p, atol=1e-10)


def test_flat_field_is_a_fair_coin():
    """No gradient: SNR = 0, the cone turns right with probability Phi(0) = 1/2."""
    g = Grid(2, 64, 64, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = np.full((64, 64), 2.0)
    n = 40000
    rng = np.random.default_rng(3)
    th = rng.uniform(0, 2 * np.pi, n)
    p = np.stack([rng.uniform(5, 58, n), rng.uniform(5, 58, n)])
    d = np.stack([np.cos(th), np.sin(th)])
    pn, dn, _ = oracle.cone_step(g, _snr_cone(snr_gain=50.0), C, 7, p, d, np.ones(n, np.uint8))
    cross = d[0] * dn[1] - d[1] * dn[0]                 # > 0: turned left (counter-clockwise)
    right = np.mean(cross < 0)
    assert abs(right - 0.5) < 4 * math.sqrt(0.25 / n)
    np.testing.assert_allclose(np.abs(cross), math.sin(TURN), atol=1e-12)   # always a full turn


def test_decisions_follow_phi_of_the_snr():
    """Many cones at one position (same C, same gradient), same heading: each turns right with
    probability Phi(SNR); their noise draws are independent (distinct cone ids)."""
    g = Grid(2, 200, 200, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = _ramp(slope=0.02)
    n = 40000
    p = np.tile(np.array([[80.0], [100.0]]), (1, n))
    th = math.pi / 2 + 0.3
    d = np.tile(np.array([[math.cos(th)], [math.sin(th)]]), (1, n))
    for gain in (5.0, 20.0, 60.0):
        c = _snr_cone(snr_gain=gain, snr_kd=3.0, snr_width=2.0)
        Cp = oracle.value_at(g, C, p[:, :1].T)[0]
        grad = oracle.gradient_at(g, C, p[:, :1].T)[0, :2]
        s = oracle.snr(c, Cp, grad, d[:, 0])
        _, dn, _ = oracle.cone_step(g, c, C, 11, p, d, np.ones(n, np.uint8))
        right = np.mean(d[0] * dn[1] - d[1] * dn[0] < 0)
        want = stats.norm.cdf(s)
        assert abs(right - want) < 4 * math.sqrt(want * (1 - want) / n) + 1e-4, (gain, s, right, want)


def test_snr_is_odd_in_the_heading_relative_to_the_gradient():
    """Mirroring the heading across the gradient direction negates the SNR; a cone heading
    along the gradient has SNR 0; the SNR is positive when the gradient lies to the right."""
    g = Grid(2, 200, 200, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = _ramp(slope=0.02)
    c = _snr_cone(snr_gain=7.0)
    Cp = oracle.value_at(g, C, [[90.0, 90.0]])[0]
    grad = oracle.gradient_at(g, C, [[90.0, 90.0]])[0, :2]
    for th in (0.3, 1.0, 2.5):
        a = oracle.snr(c, Cp, grad, [math.cos(th), math.sin(th)])
        b = oracle.snr(c, Cp, grad, [math.cos(-th), math.sin(-th)])
        assert a > 0 and b == pytest.approx(-a, rel=1e-12)
    assert oracle.snr(c, Cp, grad, [1.0, 0.0]) == pytest.approx(0.0, abs=1e-15)


def test_turn_decision_uses_the_cones_first_normal_draw():
    """The draw from N(SNR, 1) is SNR plus the cone's first normal deviate of that step, the one
    the vector-addition rule adds to its x component: cone a at step n turns right exactly when
    SNR + xi_0(seed, a, n) > 0."""
    g = Grid(2, 200, 200, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = _ramp(slope=0.02)
    n = 4000
    rng = np.random.default_rng(17)
    p = np.stack([rng.uniform(20, 180, n), rng.uniform(20, 180, n)])
    th = rng.uniform(0, 2 * np.pi, n)
    d = np.stack([np.cos(th), np.sin(th)])
    c = _snr_cone(snr_gain=20.0, snr_kd=3.0, snr_width=2.0, seed=31)
    step = 5
    _, dn, _ = oracle.cone_step(g, c, C, step, p, d, np.ones(n, np.uint8))
    right = d[0] * dn[1] - d[1] * dn[0] < 0
    xi = oracle.noise(31, np.arange(n, dtype=np.uint32), np.full(n, step, np.uint32), 2)
    Cp = oracle.value_at(g, C, p.T)
    grad = oracle.gradient_at(g, C, p.T)[:, :2]
    s = np.array([oracle.snr(c, Cp[a], grad[a], d[:, a]) for a in range(n)])
    assert 0.2 < np.mean(right) < 0.8 and np.mean(np.abs(s) < 1.5) > 0.3      # decisions not all forced
    np.testing.assert_array_equal(right, s + xi[:, 0] > 0)


def test_outside_the_window_the_cone_keeps_its_direction():
    g = Grid(2, 200, 200, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = _ramp()                                         # values 1 .. 3
    rng = np.random.default_rng(5)
    n = 500
    th = rng.uniform(0, 2 * np.pi, n)
    p = np.stack([rng.uniform(20, 180, n), rng.uniform(20, 180, n)])
    d = np.stack([np.cos(th), np.sin(th)])
    for lo, hi in ((5.0, 9.0), (0.0, 0.5)):
        c = _snr_cone(snr_gain=1e6, snr_cmin=lo, snr_cmax=hi)
        _, pos, dirs, act = oracle.run(g, c, C, 0, 20, (), (), None, p, d, np.ones(n, np.uint8))
        np.testing.assert_allclose(dirs, d, atol=1e-15)
        np.testing.assert_allclose(pos, p + 20 * 0.5 * d, atol=1e-10)


def test_vector_addition_rule_is_the_default():
    """steer = 0 ignores the SNR parameters (the pinned vector-addition step)."""
    g = Grid(2, 64, 64, h=1.0, D=0.0, lam=0.0, dt=0.2)
    C = np.random.default_rng(8).uniform(0, 1, (64, 64))
    rng = np.random.default_rng(9)
    n = 300
    p = np.stack([rng.uniform(3, 60, n), rng.uniform(3, 60, n)])
    th = rng.uniform(0, 2 * np.pi, n)
    d = np.stack([np.cos(th), np.sin(th)])
    a = oracle.cone_step(g, Cone(seed=4), C, 3, p, d, np.ones(n, np.uint8))
    b = oracle.cone_step(g, Cone(seed=4, snr_gain=99.0, snr_kd=0.1, snr_turn=1.0), C, 3, p, d,
                         np.ones(n, np.uint8))
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_snr_shape_in_concentration_steepness_and_angle():
    """Structure of Eq. 5 without restating it: linear in the gain, the cone width and |grad C|
    at fixed gamma; as a function of gamma at fixed steepness mu it rises like sqrt(gamma) from
    0 and peaks where d/dgamma [gamma / (1 + gamma)^3] = 0, i.e. at gamma = 1/2; it scales with
    the sine of the angle between heading and gradient."""
    c = _snr_cone(snr_gain=3.0, snr_width=2.0, snr_kd=4.0)
    d = [0.0, 1.0]                                        # heading +y, gradient +x: sin = 1

    def at_gamma(gamma, mu=0.05):
        Cp = gamma * c.snr_kd
        gn = mu * Cp / c.snr_width                        # |grad C| giving steepness mu
        return oracle.snr(c, Cp, [gn, 0.0], d)

    base = at_gamma(1.0)
    assert oracle.snr(_snr_cone(snr_gain=6.0, snr_width=2.0, snr_kd=4.0), 4.0, [0.1, 0.0], d) == \
        pytest.approx(2 * oracle.snr(c, 4.0, [0.1, 0.0], d), rel=1e-14)
    assert oracle.snr(c, 4.0, [0.3, 0.0], d) == pytest.approx(3 * oracle.snr(c, 4.0, [0.1, 0.0], d), rel=1e-14)
    assert oracle.snr(_snr_cone(snr_gain=3.0, snr_width=5.0, snr_kd=4.0), 4.0, [0.1, 0.0], d) == \
        pytest.approx(2.5 * oracle.snr(c, 4.0, [0.1, 0.0], d), rel=1e-14)
    assert at_gamma(0.5) > at_gamma(0.49) and at_gamma(0.5) > at_gamma(0.51)
    assert at_gamma(4e-8) / at_gamma(1e-8) == pytest.approx(2.0, rel=1e-6)
    assert base > 0
    for phi, ratio in ((math.pi / 6, 0.5), (math.pi / 4, math.sqrt(0.5))):
        gx, gy = math.cos(math.pi / 2 - phi), math.sin(math.pi / 2 - phi)   # gradient phi right of +y
        s = oracle.snr(c, 4.0, [0.1 * gx, 0.1 * gy], d)
        assert s == pytest.approx(ratio * oracle.snr(c, 4.0, [0.1, 0.0], d), rel=1e-12)


def test_cue_value_reproduces_bilinear_fields():
    """The SNR rule reads C at the tip by bilinear interpolation (Sec. 3.5): any field
    a + b x + c y + e x y is reproduced exactly between the nodes, and a node's value is
    returned at the node itself, the last row and column included."""
    nx, ny, h = 40, 30, 0.5
    g = Grid(2, nx, ny, h=h, D=0.0, lam=0.0, dt=0.2)
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    a, b, c, e = 1.5, -0.3, 0.7, 0.05
    C = a + b * x[None, :] + c * y[:, None] + e * x[None, :] * y[:, None]
    rng = np.random.default_rng(21)
    p = np.stack([rng.uniform(0, x[-1], 400), rng.uniform(0, y[-1], 400)], axis=1)
    want = a + b * p[:, 0] + c * p[:, 1] + e * p[:, 0] * p[:, 1]
    np.testing.assert_allclose(oracle.value_at(g, C, p), want, rtol=1e-13, atol=1e-13)
    corners = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (17, 9)]
    got = oracle.value_at(g, C, [(i * h, j * h) for i, j in corners])
    np.testing.assert_allclose(got, [C[j, i] for i, j in corners], rtol=1e-14)
