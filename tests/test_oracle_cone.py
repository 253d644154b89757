"""Pins of the oracle's gradient sampling, noise and cone step.

Each check compares the oracle with something fixed independently of its
code: exact gradients of linear and quadratic fields, a hand enumeration of the
interpolation corners, a scalar angle recurrence, straight lines, the normal
distribution, and an independent Philox implementation (Triton's, run by its
CPU interpreter).
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import scipy.stats

import oracle
from oracle import Cone, Grid


def _field(shape, fn):
    idx = np.indices(shape).astype(np.float64)
    if len(shape) == 2:
        y, x = idx
        return fn(x, y, 0.0)
    z, y, x = idx
    return fn(x, y, z)


# --------------------------------------------------------------- gradients
@pytest.mark.parametrize("dim,shape,h", [(2, (9, 13), 1.0), (2, (13, 9), 0.7), (3, (7, 8, 9), 1.5)])
def test_gradient_of_linear_field_is_exact(dim, shape, h):
    a, b, c = 0.37, -1.25, 2.0
    C = _field(shape, lambda x, y, z: a * x * h + b * y * h + c * z * h)
    g = Grid(dim, *shape[::-1], h=h)
    rng = np.random.default_rng(0)
    ext = np.array(shape[::-1], float)
    # interior: the 4-node footprint (i0-1 .. i0+2) stays off the walls
    p = rng.uniform(1.0, 1.0, (200, dim)) + rng.uniform(0, 1, (200, dim)) * (ext - 4)
    p *= h
    got = oracle.gradient_at(g, C, p)
    want = np.array([a, b, c])[:dim]
    np.testing.assert_allclose(got[:, :dim], np.broadcast_to(want, (200, dim)), rtol=0, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_of_quadratic_field_is_exact(dim):
    """Central differences are exact for quadratics; the node gradient is then linear and
    multilinear interpolation reproduces it exactly."""
    h = 0.5
    shape = (10, 12) if dim == 2 else (8, 9, 10)
    C = _field(shape, lambda x, y, z: (x * h) ** 2 + 3 * (y * h) ** 2 + (x * h) * (y * h)
               + 2 * (z * h) ** 2 - (x * h) * (z * h))
    g = Grid(dim, *shape[::-1], h=h)
    rng = np.random.default_rng(1)
    ext = np.array(shape[::-1], float)
    p = (1.0 + rng.uniform(0, 1, (300, dim)) * (ext - 4)) * h
    got = oracle.gradient_at(g, C, p)
    x, y = p[:, 0], p[:, 1]
    z = p[:, 2] if dim == 3 else 0 * x
    want = np.stack([2 * x + y - z, 6 * y + x, 4 * z - x], 1)
    np.testing.assert_allclose(got[:, :dim], want[:, :dim], rtol=1e-12, atol=1e-11)


def test_node_gradient_on_walls_is_half_one_sided_difference():
    rng = np.random.default_rng(2)
    C = rng.uniform(0, 1, (4, 5))
    h = 0.8
    g = Grid(2, 5, 4, h=h)
    np.testing.assert_allclose(oracle.node_gradient(g, C, 0, 2)[:2],
                               [(C[2, 1] - C[2, 0]) / (2 * h), (C[3, 0] - C[1, 0]) / (2 * h)])
    np.testing.assert_allclose(oracle.node_gradient(g, C, 4, 3)[:2],
                               [(C[3, 4] - C[3, 3]) / (2 * h), (C[3, 4] - C[2, 4]) / (2 * h)])
    np.testing.assert_allclose(oracle.node_gradient(g, C, 2, 1)[:2],
                               [(C[1, 3] - C[1, 1]) / (2 * h), (C[2, 2] - C[0, 2]) / (2 * h)])


def test_node_gradient_on_3d_walls():
    """3D: every axis takes half the one-sided difference on both of its walls and the central
    difference one node inside them (the z axis included)."""
    rng = np.random.default_rng(12)
    nx, ny, nz, h = 5, 4, 6, 0.6
    C = rng.uniform(0, 1, (nz, ny, nx))
    g = Grid(3, nx, ny, nz, h=h)
    for (i, j, k) in [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (1, 2, nz - 2), (nx - 2, 1, 1), (2, ny - 2, nz - 1)]:
        ip, im = min(i + 1, nx - 1), max(i - 1, 0)
        jp, jm = min(j + 1, ny - 1), max(j - 1, 0)
        kp, km = min(k + 1, nz - 1), max(k - 1, 0)
        want = [(C[k, j, ip] - C[k, j, im]) / (2 * h), (C[k, jp, i] - C[k, jm, i]) / (2 * h),
                (C[kp, j, i] - C[km, j, i]) / (2 * h)]
        np.testing.assert_allclose(oracle.node_gradient(g, C, i, j, k), want, rtol=1e-14, err_msg=str((i, j, k)))


def test_bilinear_corners_by_hand():
    """p = (1.25, 2.5) on a 4x5 grid: corners (1,2) (2,2) (1,3) (2,3), weights written out."""
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, (5, 4))      # ny=5, nx=4
    g = Grid(2, 4, 5, h=1.0)

    def ng(i, j):                      # node gradient, ghost = edge, written for this grid
        ip, im = min(i + 1, 3), max(i - 1, 0)
        jp, jm = min(j + 1, 4), max(j - 1, 0)
        return np.array([(C[j, ip] - C[j, im]) / 2, (C[jp, i] - C[jm, i]) / 2])

    want = (0.75 * 0.5 * ng(1, 2) + 0.25 * 0.5 * ng(2, 2)
            + 0.75 * 0.5 * ng(1, 3) + 0.25 * 0.5 * ng(2, 3))
    got = oracle.gradient_at(g, C, [[1.25, 2.5]])[0, :2]
    np.testing.assert_allclose(got, want, rtol=1e-14)
    # on the far wall the cell index is clamped to N-2 and f reaches 1
    want_edge = ng(3, 4)
    got_edge = oracle.gradient_at(g, C, [[3.0, 4.0]])[0, :2]
    np.testing.assert_allclose(got_edge, want_edge, rtol=1e-14)


# --------------------------------------------------------------- noise
def test_box_muller_noise_is_standard_normal():
    n = 1_000_000
    axon = np.arange(n, dtype=np.uint32) % 50_000
    step = (np.arange(n, dtype=np.uint32) // 50_000) * 7 + 3
    xi = oracle.noise(0x5EED0002, axon, step, 3)
    for c in range(3):
        v = xi[:, c]
        assert abs(v.mean()) < 5 / math.sqrt(n)
        assert abs(v.var() - 1) < 5 * math.sqrt(2 / n)
        assert scipy.stats.kstest(v, "norm").pvalue > 1e-3
    cc = np.corrcoef(xi.T)
    assert np.abs(cc - np.eye(3)).max() < 5 / math.sqrt(n)
    # different steps / cones / seeds draw different numbers
    assert not np.allclose(oracle.noise(1, [5], [0], 2), oracle.noise(1, [5], [1], 2))
    assert not np.allclose(oracle.noise(1, [5], [0], 2), oracle.noise(1, [6], [0], 2))
    assert not np.allclose(oracle.noise(1, [5], [0], 2), oracle.noise(1 << 32, [5], [0], 2))


def test_noise_uses_the_documented_words():
    """u1 from word 0 (in (0,1]), u2 from word 1, u3/u4 from words 2/3."""
    seed = 0xDEADBEEF12345678
    words = oracle.philox4x32_10([[17, 9, 0, 0]], [[seed & 0xFFFFFFFF, seed >> 32]])[0]
    u = [((int(words[0]) >> 8) + 1) / 2**24, (int(words[1]) >> 8) / 2**24,
         ((int(words[2]) >> 8) + 1) / 2**24, (int(words[3]) >> 8) / 2**24]
    r1, r2 = math.sqrt(-2 * math.log(u[0])), math.sqrt(-2 * math.log(u[2]))
    want = [r1 * math.cos(2 * math.pi * u[1]), r1 * math.sin(2 * math.pi * u[1]),
            r2 * math.cos(2 * math.pi * u[3])]
    np.testing.assert_allclose(oracle.noise(seed, [17], [9], 3)[0], want, rtol=1e-15, atol=1e-15)


_TRITON_PROBE = textwrap.dedent("""
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c0p, c1p, c2p, c3p, o0, o1, o2, o3, seed, N: tl.constexpr):
        o = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + o), tl.load(c1p + o), tl.load(c2p + o),
                               tl.load(c3p + o), 10)
        tl.store(o0 + o, a); tl.store(o1 + o, b); tl.store(o2 + o, c); tl.store(o3 + o, d)

    req = json.loads(sys.stdin.read())
    out = []
    for seed, ctr in req:
        ctr = np.array(ctr, dtype=np.int64)
        cs = [torch.from_numpy(ctr[:, i].copy()).to(torch.uint32) for i in range(4)]
        os_ = [torch.empty(len(ctr), dtype=torch.uint32) for _ in range(4)]
        k[(1,)](*cs, *os_, seed, N=len(ctr))
        out.append(np.stack([o.to(torch.int64).numpy() for o in os_], 1).tolist())
    print(json.dumps(out))
""")


def test_philox_matches_independent_implementation():
    """The oracle's Philox-4x32-10 equals Triton's (interpreted on the CPU) bit for bit."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    import json
    rng = np.random.default_rng(4)
    seeds = [0, 1, 0x5EED0002, 0xFFFFFFFFFFFFFFFF, int(rng.integers(0, 2**63))]
    req = []
    for s in seeds:
        ctr = rng.integers(0, 2**32, (16, 4), dtype=np.uint64)
        ctr[0] = 0
        ctr[1] = 0xFFFFFFFF
        ctr[2, 2:] = 0
        req.append([s, ctr.astype(np.int64).tolist()])
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", _TRITON_PROBE], input=json.dumps(req),
                         capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    ref = json.loads(res.stdout.strip().splitlines()[-1])
    for (s, ctr), want in zip(req, ref):
        key = np.array([[s & 0xFFFFFFFF, s >> 32]], dtype=np.uint32)
        got = oracle.philox4x32_10(np.array(ctr, dtype=np.uint32), key)
        np.testing.assert_array_equal(got.astype(np.int64), np.array(want, dtype=np.int64))


# --------------------------------------------------------------- cone step
def _one(dim, p, d):
    return (np.array(p, float).reshape(dim, 1), np.array(d, float).reshape(dim, 1),
            np.ones(1, np.uint8))


@pytest.mark.parametrize("dim", [2, 3])
def test_straight_line_without_cue_or_noise(dim):
    shape = (40, 50) if dim == 2 else (30, 32, 34)
    g = Grid(dim, *shape[::-1], h=1.0)
    rng = np.random.default_rng(5)
    C = rng.uniform(0, 1, shape)
    d = rng.standard_normal(dim)
    d /= np.linalg.norm(d)
    p0 = np.array(shape[::-1], float)[:dim] / 2
    n = 12
    cone = Cone(w_prev=0.7, w_grad=0.0, w_noise=0.0, step_len=0.5)
    pos, dirs, act = _one(dim, p0, d)
    for s in range(n):
        pos, dirs, act = oracle.cone_step(g, cone, C, s, pos, dirs, act)
    np.testing.assert_allclose(pos[:, 0], p0 + n * 0.5 * d, rtol=0, atol=1e-12)
    np.testing.assert_allclose(dirs[:, 0], d, atol=1e-14)
    assert act[0] == 1


def test_angle_follows_scalar_recurrence_in_a_linear_field():
    """w_n = 0 and a linear field: ghat is constant (+x), and the heading obeys
    theta' = atan2(w_p sin theta, w_p cos theta + w_g)."""
    shape = (200, 300)
    g = Grid(2, 300, 200, h=1.0)
    C = _field(shape, lambda x, y, z: 0.01 * x)
    wp, wg = 0.5, 0.4
    cone = Cone(w_prev=wp, w_grad=wg, w_noise=0.0, step_len=0.5)
    th = 2.5
    pos, dirs, act = _one(2, [150.0, 100.0], [math.cos(th), math.sin(th)])
    p = np.array([150.0, 100.0])
    for s in range(30):
        pos, dirs, act = oracle.cone_step(g, cone, C, s, pos, dirs, act)
        th = math.atan2(wp * math.sin(th), wp * math.cos(th) + wg)
        p = p + 0.5 * np.array([math.cos(th), math.sin(th)])
        assert abs(math.atan2(dirs[1, 0], dirs[0, 0]) - th) < 1e-12
    np.testing.assert_allclose(pos[:, 0], p, atol=1e-10)


def test_gradient_sign_turns_cone_up_the_cue():
    """A cone moving along +y in a field rising along -x turns toward -x."""
    g = Grid(2, 60, 60)
    C = _field((60, 60), lambda x, y, z: 5.0 - 0.05 * x)
    cone = Cone(w_prev=0.5, w_grad=0.4, w_noise=0.0)
    pos, dirs, act = _one(2, [30.0, 30.0], [0.0, 1.0])
    pos, dirs, act = oracle.cone_step(g, cone, C, 0, pos, dirs, act)
    assert dirs[0, 0] < -0.5 and dirs[1, 0] > 0


def test_zero_gradient_and_zero_blend():
    g = Grid(2, 20, 20)
    C = np.full((20, 20), 3.0)
    # constant field: ghat = 0, so with no noise the heading is kept
    pos, dirs, act = oracle.cone_step(g, Cone(w_noise=0.0), C, 0, *_one(2, [10, 10], [0.6, 0.8]))
    np.testing.assert_allclose(dirs[:, 0], [0.6, 0.8], atol=1e-15)
    np.testing.assert_allclose(pos[:, 0], [10.3, 10.4], atol=1e-14)
    # all weights zero: |v| = 0, the previous direction is kept
    pos, dirs, act = oracle.cone_step(g, Cone(w_prev=0, w_grad=0, w_noise=0), C, 0,
                                      *_one(2, [10, 10], [0.6, 0.8]))
    np.testing.assert_allclose(dirs[:, 0], [0.6, 0.8], atol=1e-15)
    # a gradient below eps is treated as zero
    Cs = _field((20, 20), lambda x, y, z: 1e-18 * x)
    pos, dirs, act = oracle.cone_step(g, Cone(w_prev=0.5, w_grad=0.4, w_noise=0.0), Cs, 0,
                                      *_one(2, [10, 10], [0.0, 1.0]))
    np.testing.assert_allclose(dirs[:, 0], [0.0, 1.0], atol=1e-15)


def test_wall_stop_keeps_last_state_and_clamp_mode_clamps():
    g = Grid(2, 10, 10)
    C = np.zeros((10, 10))
    cone = Cone(w_noise=0.0, step_len=0.5)
    # 0.3 from the right wall (x = 9), heading +x: leaves the domain
    pos, dirs, act = oracle.cone_step(g, cone, C, 0, *_one(2, [8.7, 4.0], [1.0, 0.0]))
    assert act[0] == 0
    np.testing.assert_allclose(pos[:, 0], [8.7, 4.0])
    # inactive cones do not move
    pos2, dirs2, act2 = oracle.cone_step(g, cone, C, 1, pos, dirs, act)
    np.testing.assert_array_equal(pos2, pos)
    # exactly on the wall is inside the domain
    pos, dirs, act = oracle.cone_step(g, cone, C, 0, *_one(2, [8.5, 4.0], [1.0, 0.0]))
    assert act[0] == 1 and pos[0, 0] == 9.0
    # clamp mode: coordinate clamped, direction kept, still active
    clamp = Cone(w_noise=0.0, step_len=0.5, wall_mode=1)
    pos, dirs, act = oracle.cone_step(g, clamp, C, 0, *_one(2, [8.7, 0.2], [0.6, -0.8]))
    assert act[0] == 1
    np.testing.assert_allclose(pos[:, 0], [9.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(dirs[:, 0], [0.6, -0.8], atol=1e-15)


def test_source_radius_stop_after_move():
    g = Grid(2, 23, 14)                 # non-square: a swapped x/y decode misses the source
    C = np.zeros((14, 23))
    src = [12 + 23 * 10]                # node (12, 10)
    cone = Cone(w_noise=0.0, step_len=0.5, stop_radius=2.0)
    # at distance 2.4 heading straight at the source: after the move 1.9 <= 2
    pos, dirs, act = oracle.cone_step(g, cone, C, 0, *_one(2, [9.6, 10.0], [1.0, 0.0]), src)
    assert act[0] == 0
    np.testing.assert_allclose(pos[:, 0], [10.1, 10.0])
    # at distance 2.6: after the move 2.1 > 2, still active
    pos, dirs, act = oracle.cone_step(g, cone, C, 0, *_one(2, [9.4, 10.0], [1.0, 0.0]), src)
    assert act[0] == 1
    # landing exactly on the radius (every quantity exact in binary): the test is inclusive
    exact = Cone(w_prev=1.0, w_grad=0.0, w_noise=0.0, step_len=0.5, stop_radius=2.0)
    pos, dirs, act = oracle.cone_step(g, exact, C, 0, *_one(2, [9.5, 10.0], [1.0, 0.0]), src)
    np.testing.assert_array_equal(pos[:, 0], [10.0, 10.0])
    assert act[0] == 0
    # 3D: node index -> coordinates uses x fastest, then y, then z
    g3 = Grid(3, 6, 7, 8)
    cell = 4 + 6 * (5 + 7 * 3)          # node (4, 5, 3)
    pos, dirs, act = oracle.cone_step(g3, cone, np.zeros((8, 7, 6)), 0,
                                      *_one(3, [4.0, 5.0, 1.4], [0.0, 0.0, 1.0]), [cell])
    assert act[0] == 0


def test_cones_read_the_field_of_their_own_step():
    """run(): the cone step of step n sees C^n.  With C^0 = 0 the first turn is absent."""
    g = Grid(2, 30, 30, D=1.0, lam=0.0, dt=0.2)
    cone = Cone(w_noise=0.0)
    src = [16 + 30 * 15]
    C, pos, dirs, act = oracle.run(g, cone, np.zeros((30, 30)), 0, 1, src, [1.0],
                                   None, np.array([[15.0], [15.0]]), np.array([[0.0], [1.0]]),
                                   np.ones(1, np.uint8))
    np.testing.assert_allclose(dirs[:, 0], [0.0, 1.0])
    C, pos, dirs, act = oracle.run(g, cone, C, 1, 1, src, [1.0], None, pos, dirs, act)
    assert dirs[0, 0] > 0.1         # now the source at +x attracts it


@pytest.mark.parametrize("dim", [2, 3])
def test_cone_paths_mirror_with_the_field(dim):
    shape = (24, 31) if dim == 2 else (12, 14, 15)
    ext = np.array(shape[::-1], float)
    g = Grid(dim, *shape[::-1], h=1.0)
    rng = np.random.default_rng(8)
    C = _field(shape, lambda x, y, z: np.exp(-((x - 9) ** 2 + (y - 7) ** 2 + (z - 5) ** 2) / 40))
    n = 20
    pos = (2 + rng.uniform(0, 1, (dim, n)) * (ext[:, None] - 5))
    d = rng.standard_normal((dim, n))
    d /= np.linalg.norm(d, axis=0)
    act = np.ones(n, np.uint8)
    cone = Cone(w_noise=0.0, step_len=0.3)
    for ax in range(dim):          # ax in x, y, z order
        base = (pos, d, act)
        mir = (pos.copy(), d.copy(), act.copy())
        mir[0][ax] = (ext[ax] - 1) - mir[0][ax]
        mir[1][ax] = -mir[1][ax]
        Cm = np.flip(C, dim - 1 - ax)
        for s in range(6):
            base = oracle.cone_step(g, cone, C, s, *base)
            mir = oracle.cone_step(g, cone, Cm, s, *mir)
        back = mir[0].copy()
        back[ax] = (ext[ax] - 1) - back[ax]
        np.testing.assert_allclose(back, base[0], atol=1e-11)
        np.testing.assert_array_equal(mir[2], base[2])
