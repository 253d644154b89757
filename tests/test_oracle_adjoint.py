"""Pins of the oracle's hand-derived adjoint: central finite differences of the
forward endpoint loss (FP64), a linear-in-sources check, and the reverse-mode
dot-product identity on the field operator."""
import numpy as np
import pytest

import oracle
from oracle import Cone, Grid


def _problem(dim, seed=0, T=30, h=1.0):
    """D scales with h^2, so alpha = D dt / h^2 (and stability) does not depend on h."""
    rng = np.random.default_rng(seed)
    if dim == 2:
        nx, ny, nz = 17, 13, 1
        shape = (ny, nx)
        g = Grid(2, nx, ny, h=h, D=0.9 * h * h, lam=0.02, dt=0.2)
    else:
        nx, ny, nz = 9, 8, 7
        shape = (nz, ny, nx)
        g = Grid(3, nx, ny, nz, h=h, D=0.8 * h * h, lam=0.03, dt=0.15)
    n_cells = int(np.prod(shape))
    cells = rng.choice(n_cells, 3, replace=False).astype(np.int32)
    emit = rng.uniform(0.5, 2.0, 3)
    smap = rng.uniform(0.0, 0.2, shape)
    C0 = rng.uniform(0.0, 1.0, shape)
    n = 6
    ext = np.array((nx, ny, nz)[:dim], float)
    pos = (1.5 + rng.uniform(0, 1, (dim, n)) * (ext[:, None] - 3)) * h
    d = rng.standard_normal((dim, n))
    d /= np.linalg.norm(d, axis=0)
    tg = rng.uniform(0, 1, (dim, n)) * (ext[:, None] - 1) * h
    c = Cone(w_prev=0.5, w_grad=0.4, w_noise=0.1, step_len=0.5 * h, stop_radius=0.0, wall_mode=1, seed=77)
    return g, c, C0, cells, emit, smap, pos, d, tg, T


def _loss(g, c, C0, cells, emit, smap, pos, d, tg, T):
    return oracle.endpoint_loss(g, c, C0, cells, emit, smap, pos, d, tg, T)


@pytest.mark.parametrize("dim,h", [(2, 1.0), (3, 1.0), (2, 0.7), (3, 1.3)])
def test_adjoint_matches_central_differences(dim, h):
    g, c, C0, cells, emit, smap, pos, d, tg, T = _problem(dim, h=h)
    loss, gD, gl, gsrc, gmap = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T)
    assert loss == pytest.approx(_loss(g, c, C0, cells, emit, smap, pos, d, tg, T), rel=1e-14)

    def fd(f, x0, h):
        return (f(x0 + h) - f(x0 - h)) / (2 * h)

    def with_grid(**kw):
        gg = Grid(g.dim, g.nx, g.ny, g.nz, h=g.h, D=kw.get("D", g.D), lam=kw.get("lam", g.lam), dt=g.dt)
        return _loss(gg, c, C0, cells, emit, smap, pos, d, tg, T)

    dD = fd(lambda x: with_grid(D=x), g.D, 1e-6)
    dl = fd(lambda x: with_grid(lam=x), g.lam, 1e-7)
    assert gD == pytest.approx(dD, rel=1e-5, abs=1e-9)
    assert gl == pytest.approx(dl, rel=1e-5, abs=1e-9)
    for k in range(len(emit)):
        def f(x, k=k):
            e = emit.copy()
            e[k] = x
            return _loss(g, c, C0, cells, e, smap, pos, d, tg, T)
        assert gsrc[k] == pytest.approx(fd(f, emit[k], 1e-6), rel=1e-5, abs=1e-9)
    rng = np.random.default_rng(5)
    for flat in rng.choice(smap.size, 6, replace=False):
        def f(x, flat=flat):
            m = smap.copy()
            m.flat[flat] = x
            return _loss(g, c, C0, cells, emit, m, pos, d, tg, T)
        assert gmap.flat[flat] == pytest.approx(fd(f, smap.flat[flat], 1e-6), rel=1e-5, abs=1e-9)


def test_source_and_map_gradients_agree_where_they_coincide():
    """A point source adds e per step, a map adds dt*M per step: at the same node,
    dL/de = dL/dM / dt exactly (both are sums of the same adjoint field)."""
    g, c, C0, cells, emit, smap, pos, d, tg, T = _problem(2, seed=3)
    loss, gD, gl, gsrc, gmap = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T)
    for k, cell in enumerate(cells):
        assert gsrc[k] == pytest.approx(gmap.flat[cell] / g.dt, rel=1e-12)


def test_no_gradient_weight_means_no_parameter_gradient():
    """w_grad = 0: the cones never read the field, so every parameter gradient vanishes."""
    g, c, C0, cells, emit, smap, pos, d, tg, T = _problem(2, seed=4)
    c0 = Cone(w_prev=0.5, w_grad=0.0, w_noise=0.1, step_len=0.5, wall_mode=1, seed=77)
    loss, gD, gl, gsrc, gmap = oracle.adjoint(g, c0, C0, cells, emit, smap, pos, d, tg, T)
    assert gD == 0.0 and gl == 0.0
    assert np.all(gsrc == 0.0) and np.all(gmap == 0.0)


def test_binary32_storage_knob_only_rounds_the_stored_states():
    """``state_binary32`` (a measuring knob) leaves the oracle proper untouched, and moves
    a well-conditioned gradient by no more than binary32 rounding of the states can."""
    g, c, C0, cells, emit, smap, pos, d, tg, T = _problem(2, seed=5)
    a = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T)
    b = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T, state_binary32=False)
    r = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T, state_binary32=True)
    assert a[0] == b[0] and a[1] == b[1] and np.array_equal(a[4], b[4])
    assert r[0] != a[0]
    assert r[0] == pytest.approx(a[0], rel=1e-5)
    assert r[1] == pytest.approx(a[1], rel=1e-3)
    # with states already in binary32 and exactly representable steps the knob changes nothing
    c_still = Cone(w_prev=1.0, w_grad=0.0, w_noise=0.0, step_len=0.5, wall_mode=1, seed=77)
    d_axis = np.zeros_like(d)
    d_axis[0] = 1.0
    pos32 = np.round(pos * 4) / 4
    C0z = np.zeros_like(C0)
    x = oracle.adjoint(g, c_still, C0z, cells[:0], emit[:0], np.zeros_like(smap), pos32, d_axis, tg, T)
    y = oracle.adjoint(g, c_still, C0z, cells[:0], emit[:0], np.zeros_like(smap), pos32, d_axis, tg, T,
                       state_binary32=True)
    assert x[0] == y[0]


@pytest.mark.parametrize("dim", [2, 3])
def test_backward_over_given_states_equals_the_full_adjoint(dim):
    """The backward pass alone (``adjoint_from_states``), fed states gathered one step at a
    time by the plain forward (``oracle.run``, not the adjoint's own storing loop), returns
    exactly the full adjoint's loss and gradients: the state layout (T + 1, dim, n) and the
    step indexing of the stored states are the ones the backward reads."""
    g, c, C0, cells, emit, smap, pos, d, tg, T = _problem(dim, seed=8, T=25)
    full = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T)
    n = pos.shape[1]
    Cs, Ps, Ds = [C0.copy()], [pos.copy()], [d.copy()]
    C, p, dd, act = C0.copy(), pos.copy(), d.copy(), np.ones(n, np.uint8)
    for s in range(T):
        C, p, dd, act = oracle.run(g, c, C, s, 1, cells, emit, smap, p, dd, act)
        Cs.append(C)
        Ps.append(p)
        Ds.append(dd)
    assert act.all()
    part = oracle.adjoint_from_states(g, c, cells, tg, np.stack(Cs), np.stack(Ps), np.stack(Ds))
    assert part[0] == full[0] and part[1] == full[1] and part[2] == full[2]
    np.testing.assert_array_equal(part[3], full[3])
    np.testing.assert_array_equal(part[4], full[4])


def test_backward_over_given_states_follows_the_states_it_is_given():
    """Fed states of another run (here: the forward stored in binary32 by hand), the backward
    pass returns the ``state_binary32`` adjoint, not the oracle's own: it reads only the states
    it is given, and its loss is the given endpoint's."""
    g, c, C0, cells, emit, smap, pos, d, tg, T = _problem(2, seed=9, T=20)
    n = pos.shape[1]
    Cs, Ps, Ds = [C0.copy()], [pos.copy()], [d.copy()]
    C, p, dd, act = C0.copy(), pos.copy(), d.copy(), np.ones(n, np.uint8)
    for s in range(T):
        C, p, dd, act = oracle.run(g, c, C, s, 1, cells, emit, smap, p, dd, act)
        C, p, dd = (x.astype(np.float32).astype(np.float64) for x in (C, p, dd))
        Cs.append(C)
        Ps.append(p)
        Ds.append(dd)
    part = oracle.adjoint_from_states(g, c, cells, tg, np.stack(Cs), np.stack(Ps), np.stack(Ds))
    r32 = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T, state_binary32=True)
    own = oracle.adjoint(g, c, C0, cells, emit, smap, pos, d, tg, T)
    assert part[0] == r32[0] and part[1] == r32[1] and part[2] == r32[2]
    np.testing.assert_array_equal(part[4], r32[4])
    assert part[1] != own[1]
    e = np.stack(Ps)[-1] - tg
    assert part[0] == pytest.approx(float((e * e).sum()) / n, rel=1e-15)
