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
