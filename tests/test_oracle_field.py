"""Pins of the oracle's field step against what the model and mathematics fix.

None of these checks re-types the oracle's loop: each compares it with a
hand enumeration, an exact invariant, a closed form, or a library solve.
"""
import numpy as np
import pytest
import scipy.fft

import oracle
from oracle import Grid

pytestmark = pytest.mark.filterwarnings("ignore")


# --------------------------------------------------------------- brute force
# 3x3 grid, every node's axis neighbours written out by hand as (i, j) lists.
NBRS_3x3 = {
    (0, 0): [(1, 0), (0, 1)],
    (1, 0): [(0, 0), (2, 0), (1, 1)],
    (2, 0): [(1, 0), (2, 1)],
    (0, 1): [(0, 0), (1, 1), (0, 2)],
    (1, 1): [(0, 1), (2, 1), (1, 0), (1, 2)],
    (2, 1): [(2, 0), (1, 1), (2, 2)],
    (0, 2): [(0, 1), (1, 2)],
    (1, 2): [(1, 1), (0, 2), (2, 2)],
    (2, 2): [(2, 1), (1, 2)],
}

# 4 wide x 2 high: non-square, so a transposed index shows up.
NBRS_4x2 = {
    (0, 0): [(1, 0), (0, 1)],
    (1, 0): [(0, 0), (2, 0), (1, 1)],
    (2, 0): [(1, 0), (3, 0), (2, 1)],
    (3, 0): [(2, 0), (3, 1)],
    (0, 1): [(0, 0), (1, 1)],
    (1, 1): [(1, 0), (0, 1), (2, 1)],
    (2, 1): [(2, 0), (1, 1), (3, 1)],
    (3, 1): [(3, 0), (2, 1)],
}


@pytest.mark.parametrize("nbrs,nx,ny", [(NBRS_3x3, 3, 3), (NBRS_4x2, 4, 2)])
def test_brute_force_single_step_2d(nbrs, nx, ny):
    rng = np.random.default_rng(11)
    C = rng.uniform(0.0, 2.0, (ny, nx))
    D, dt, h, lam = 0.7, 0.3, 1.3, 0.05
    alpha = D * dt / h**2
    src_cell = [nx + 1, 0]          # node (1,1) and node (0,0)
    src_emit = [0.25, 1.5]
    expected = np.empty_like(C)
    for (i, j), lst in nbrs.items():
        flux = sum(C[jj, ii] - C[j, i] for (ii, jj) in lst)
        expected[j, i] = C[j, i] + alpha * flux - lam * dt * C[j, i]
    expected[1, 1] += 0.25
    expected[0, 0] += 1.5
    got = oracle.field_step(Grid(2, nx, ny, h=h, D=D, lam=lam, dt=dt), C, src_cell, src_emit)
    np.testing.assert_allclose(got, expected, rtol=0, atol=1e-14)


def test_brute_force_single_step_3d():
    # 3x2x2 grid; neighbours listed by hand for every node as (i, j, k).
    nbrs = {
        (0, 0, 0): [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
        (1, 0, 0): [(0, 0, 0), (2, 0, 0), (1, 1, 0), (1, 0, 1)],
        (2, 0, 0): [(1, 0, 0), (2, 1, 0), (2, 0, 1)],
        (0, 1, 0): [(1, 1, 0), (0, 0, 0), (0, 1, 1)],
        (1, 1, 0): [(0, 1, 0), (2, 1, 0), (1, 0, 0), (1, 1, 1)],
        (2, 1, 0): [(1, 1, 0), (2, 0, 0), (2, 1, 1)],
        (0, 0, 1): [(1, 0, 1), (0, 1, 1), (0, 0, 0)],
        (1, 0, 1): [(0, 0, 1), (2, 0, 1), (1, 1, 1), (1, 0, 0)],
        (2, 0, 1): [(1, 0, 1), (2, 1, 1), (2, 0, 0)],
        (0, 1, 1): [(1, 1, 1), (0, 0, 1), (0, 1, 0)],
        (1, 1, 1): [(0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 1, 0)],
        (2, 1, 1): [(1, 1, 1), (2, 0, 1), (2, 1, 0)],
    }
    rng = np.random.default_rng(12)
    nx, ny, nz = 3, 2, 2
    C = rng.uniform(0.0, 2.0, (nz, ny, nx))
    D, dt, h, lam = 0.5, 0.2, 1.0, 0.1
    alpha = D * dt / h**2
    expected = np.empty_like(C)
    for (i, j, k), lst in nbrs.items():
        flux = sum(C[kk, jj, ii] - C[k, j, i] for (ii, jj, kk) in lst)
        expected[k, j, i] = C[k, j, i] + alpha * flux - lam * dt * C[k, j, i]
    expected[1, 0, 2] += 0.75       # node (2,0,1) = 2 + 3*(0 + 2*1) = 8
    smap = rng.uniform(0, 1, C.shape)
    expected += dt * smap
    got = oracle.field_step(Grid(3, nx, ny, nz, h=h, D=D, lam=lam, dt=dt), C, [8], [0.75], smap)
    np.testing.assert_allclose(got, expected, rtol=0, atol=1e-14)


# --------------------------------------------------------------- invariants
@pytest.mark.parametrize("dim,shape", [(2, (37, 23)), (3, (9, 11, 7))])
def test_mass_conservation_no_flux(dim, shape):
    """lambda = 0 and no-flux walls: sum C^n = sum C^0 + n * sum e_k exactly."""
    rng = np.random.default_rng(1)
    C = rng.uniform(0, 1, shape)
    n_cells = C.size
    cells = rng.choice(n_cells, 5, replace=False)
    emit = rng.uniform(0.5, 2.0, 5)
    ext = shape[::-1]
    g = Grid(dim, *ext, D=1.0, lam=0.0, dt=0.15 if dim == 3 else 0.2)
    m0 = C.sum()
    n = 60
    Cn, *_ = oracle.run(g, oracle.Cone(), C, 0, n, cells, emit)
    assert abs(Cn.sum() - (m0 + n * emit.sum())) <= 1e-12 * (m0 + n * emit.sum())
    # and the wall-adjacent nodes received mass: the field is not simply clipped
    assert Cn.min() > 0


def _moments(C, h):
    idx = np.indices(C.shape).astype(np.float64) * h   # axis order (z,) y, x
    m = C.sum()
    mean = [(x * C).sum() / m for x in idx]
    var = [(((x - mu) ** 2) * C).sum() / m for x, mu in zip(idx, mean)]
    return m, mean, var


@pytest.mark.parametrize("dim,shape,h,D,dt,lam", [
    (2, (41, 61), 1.0, 1.0, 0.2, 0.0),
    (2, (61, 41), 0.5, 0.25, 0.3, 0.03),
    (3, (25, 31, 27), 1.0, 1.0, 0.15, 0.0),
    (3, (27, 25, 31), 2.0, 3.0, 0.2, 0.01),
])
def test_discrete_variance_growth(dim, shape, h, D, dt, lam):
    """An impulse spreads with per-axis variance exactly 2 D dt n / (1 - lambda dt) (FTCS,
    before it meets a wall): the neighbour-difference sum adds 2 alpha h^2 times the mass to
    the second moment each step while decay scales moment and mass alike."""
    C = np.zeros(shape)
    centre = tuple(s // 2 for s in shape)
    C[centre] = 3.0
    g = Grid(dim, *shape[::-1], h=h, D=D, lam=lam, dt=dt)
    n = min(shape) // 2 - 1      # support grows by one node per step
    Cn, *_ = oracle.run(g, oracle.Cone(), C, 0, n)
    m, mean, var = _moments(Cn, h)
    assert abs(m - 3.0 * (1 - lam * dt) ** n) < 1e-12
    for ax in range(dim):
        assert abs(mean[ax] - centre[ax] * h) < 1e-10
        want = 2.0 * D * n * dt / (1.0 - lam * dt)
        assert abs(var[ax] - want) < 1e-9 * want


@pytest.mark.parametrize("dim", [2, 3])
def test_heat_kernel(dim):
    """Far from walls the impulse response approaches the Gaussian heat kernel, O(h^2/(D t))."""
    N = 121 if dim == 2 else 61
    shape = (N,) * dim
    M = 1.0
    C = np.zeros(shape)
    c = N // 2
    C[(c,) * dim] = M
    dt = 0.2 if dim == 2 else 0.15
    g = Grid(dim, *shape, h=1.0, D=1.0, lam=0.0, dt=dt)
    r2 = sum((x - c) ** 2 for x in np.indices(shape).astype(float))
    errs = []
    steps = [50, 100, 200] if dim == 2 else [40, 80, 160]
    Ccur, done = C, 0
    for n in steps:
        Ccur, *_ = oracle.run(g, oracle.Cone(), Ccur, 0, n - done)
        done = n
        t = n * dt
        kern = M * (4 * np.pi * t) ** (-dim / 2) * np.exp(-r2 / (4 * t))
        errs.append(np.abs(Ccur - kern).max() / kern.max())
    assert errs[0] < 0.05
    assert errs[2] < errs[1] < errs[0]


# --------------------------------------------------------------- closed forms
def test_pure_decay_closed_form():
    """D = 0: C^n = q^n C^0 + e (1 - q^n)/(lambda dt) at sources, q = 1 - lambda dt."""
    g = Grid(2, 7, 5, D=0.0, lam=0.03, dt=0.25)
    C = np.full((5, 7), 2.0)
    cells = [3, 17]
    emit = [0.5, 1.25]
    n = 37
    Cn, *_ = oracle.run(g, oracle.Cone(), C, 0, n, cells, emit)
    q = 1 - g.lam * g.dt
    want = np.full((5, 7), 2.0 * q**n)
    for c, e in zip(cells, emit):
        want.flat[c] += e * (1 - q**n) / (g.lam * g.dt)
    np.testing.assert_allclose(Cn, want, rtol=1e-13)


def _dct_steady_state(shape, alpha, decay, rhs):
    """Solve (decay I - alpha L) C = rhs with L the no-flux node Laplacian, by DCT-II."""
    lam_sum = np.zeros(shape)
    for ax, n in enumerate(shape):
        k = np.arange(n)
        ev = 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2
        sh = [1] * len(shape)
        sh[ax] = n
        lam_sum = lam_sum + ev.reshape(sh)
    rh = scipy.fft.dctn(rhs, type=2, norm="ortho")
    return scipy.fft.idctn(rh / (decay + alpha * lam_sum), type=2, norm="ortho")


@pytest.mark.parametrize("dim,shape,h,D,dt,lam,with_map", [
    (2, (17, 24), 1.0, 1.0, 0.2, 0.1, False),
    (2, (24, 17), 0.5, 0.25, 0.2, 0.15, True),
    (3, (6, 7, 8), 1.0, 1.0, 0.15, 0.2, False),
    (3, (8, 6, 7), 1.0, 0.5, 0.2, 0.1, True),
])
def test_steady_state_matches_dct_solve(dim, shape, h, D, dt, lam, with_map):
    rng = np.random.default_rng(3)
    n_cells = int(np.prod(shape))
    cells = rng.choice(n_cells, 3, replace=False)
    emit = rng.uniform(0.5, 2.0, 3)
    smap = rng.uniform(0, 1, shape) if with_map else None
    g = Grid(dim, *shape[::-1], h=h, D=D, lam=lam, dt=dt)
    q = 1 - lam * dt
    nsteps = int(np.ceil(np.log(1e-14) / np.log(q)))
    C, *_ = oracle.run(g, oracle.Cone(), np.zeros(shape), 0, nsteps, cells, emit, smap)
    rhs = np.zeros(shape)
    for c, e in zip(cells, emit):
        rhs.flat[c] += e
    if with_map:
        rhs += dt * smap
    want = _dct_steady_state(shape, D * dt / h**2, lam * dt, rhs)
    np.testing.assert_allclose(C, want, rtol=1e-10, atol=1e-12 * want.max())


# --------------------------------------------------------------- symmetries
@pytest.mark.parametrize("dim,shape", [(2, (13, 20)), (3, (6, 9, 11))])
def test_mirror_symmetry(dim, shape):
    rng = np.random.default_rng(5)
    C0 = rng.uniform(0, 1, shape)
    n_cells = C0.size
    cells = rng.choice(n_cells, 4, replace=False)
    emit = rng.uniform(0.5, 2, 4)
    g = Grid(dim, *shape[::-1], D=0.8, lam=0.02, dt=0.2 if dim == 2 else 0.15)
    base, *_ = oracle.run(g, oracle.Cone(), C0, 0, 25, cells, emit)
    for ax in range(dim):
        coords = np.array(np.unravel_index(cells, shape))
        coords[ax] = shape[ax] - 1 - coords[ax]
        mcells = np.ravel_multi_index(tuple(coords), shape)
        mir, *_ = oracle.run(g, oracle.Cone(), np.flip(C0, ax), 0, 25, mcells, emit)
        np.testing.assert_allclose(mir, np.flip(base, ax), rtol=1e-14, atol=1e-14)


def test_transpose_symmetry_square():
    rng = np.random.default_rng(6)
    C0 = rng.uniform(0, 1, (15, 15))
    g = Grid(2, 15, 15, D=1.0, lam=0.01, dt=0.2)
    cells = np.array([3 + 15 * 7, 11 + 15 * 2])
    emit = np.array([1.0, 0.7])
    base, *_ = oracle.run(g, oracle.Cone(), C0, 0, 30, cells, emit)
    tcells = (cells // 15) + 15 * (cells % 15)
    tr, *_ = oracle.run(g, oracle.Cone(), C0.T, 0, 30, tcells, emit)
    np.testing.assert_allclose(tr, base.T, rtol=1e-14, atol=1e-14)


def _apply_L(shape, x):
    """L_h x recovered from one step with alpha = 1, no decay, no sources."""
    dim = len(shape)
    g = Grid(dim, *shape[::-1], h=1.0, D=1.0, lam=0.0, dt=1.0)
    return oracle.field_step(g, x) - x


@pytest.mark.parametrize("shape", [(9, 14), (5, 6, 7)])
def test_laplacian_self_adjoint_and_kills_constants(shape):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(shape)
    y = rng.standard_normal(shape)
    lhs = (_apply_L(shape, x) * y).sum()
    rhs = (x * _apply_L(shape, y)).sum()
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)
    assert np.abs(_apply_L(shape, np.full(shape, 3.7))).max() < 1e-15
    # negative semi-definite: <x, L x> <= 0 (diffusion never creates variance)
    assert (x * _apply_L(shape, x)).sum() < 0


@pytest.mark.parametrize("dim", [2, 3])
def test_threaded_field_step_is_the_single_threaded_one(dim):
    """The timed CPU baseline may split the field's node loop over threads; every node's
    update reads only the old field, so the result must not change by a single bit."""
    rng = np.random.default_rng(11 + dim)
    if dim == 2:
        g = oracle.Grid(2, 97, 61, h=1.0, D=1.0, lam=0.01, dt=0.2)
    else:
        g = oracle.Grid(3, 23, 17, 13, h=1.0, D=1.0, lam=0.01, dt=0.15)
    C = rng.uniform(0.0, 1.0, g.shape)
    cells = rng.choice(C.size, 5, replace=False)
    emit = rng.uniform(0.5, 2.0, 5)
    smap = rng.uniform(0.0, 1.0, g.shape)
    try:
        oracle.set_threads(4)
        a = oracle.field_step(g, C, cells, emit, smap)
    finally:
        oracle.set_threads(1)
    b = oracle.field_step(g, C, cells, emit, smap)
    np.testing.assert_array_equal(a, b)


def _padded_window(C, origin, size):
    """The input values of a window grown by one node on every side; nodes outside the grid
    are NaN (the windowed step must never read them)."""
    dim = C.ndim
    shape_pad = tuple(s + 2 for s in reversed(size))             # (z,) y, x order
    Wp = np.full(shape_pad, np.nan)
    lo = [o - 1 for o in origin]
    ext = list(reversed(C.shape))                                 # x, y(, z)
    for idx in np.ndindex(*shape_pad):
        g = [lo[a] + idx[dim - 1 - a] for a in range(dim)]       # global x, y(, z)
        if all(0 <= g[a] < ext[a] for a in range(dim)):
            Wp[idx] = C[tuple(reversed(g))]
    return Wp


@pytest.mark.parametrize("dim", [2, 3])
def test_windowed_field_step_equals_the_full_step(dim):
    """The windowed form of the field step (used to check grids too large for the oracle)
    gives, on corner, edge and interior windows, exactly the full step's values there, and
    never reads outside the grid (those entries are NaN)."""
    rng = np.random.default_rng(40 + dim)
    if dim == 2:
        g = oracle.Grid(2, 37, 29, h=1.0, D=1.0, lam=0.01, dt=0.2)
        windows = [((0, 0), (5, 4)), ((32, 25), (5, 4)), ((10, 0), (7, 3)), ((0, 11), (3, 6)), ((12, 9), (8, 8))]
    else:
        g = oracle.Grid(3, 13, 11, 9, h=1.0, D=1.0, lam=0.01, dt=0.15)
        windows = [((0, 0, 0), (4, 3, 2)), ((9, 8, 7), (4, 3, 2)), ((5, 0, 3), (3, 2, 4)), ((4, 4, 4), (5, 5, 3))]
    C = rng.uniform(0.0, 1.0, g.shape)
    cells = rng.choice(C.size, 6, replace=False)
    cells[0] = 0
    cells[1] = C.size - 1
    emit = rng.uniform(0.5, 2.0, 6)
    full = oracle.field_step(g, C, cells, emit)
    for origin, size in windows:
        got = oracle.field_window(g, _padded_window(C, origin, size), origin, cells, emit)
        sl = tuple(slice(o, o + s) for o, s in zip(reversed(origin), reversed(size)))
        np.testing.assert_array_equal(got, full[sl])


@pytest.mark.parametrize("dim", [2, 3])
def test_steady_state_follows_the_continuum_greens_function(dim):
    """A point source emitting e per step, run to its steady state on a grid whose walls lie
    many screening lengths l = sqrt(D / lambda) away: a few nodes from the source the field
    follows the free-space solution of D lap C - lambda C = -(e / dt) delta, namely
    (e/dt) / (2 pi D) K0(r / l) in 2D and (e/dt) / (4 pi D r) exp(-r / l) in 3D, to the
    discretisation error of the 5- / 7-point operator, which shrinks away from the source."""
    from scipy.special import k0
    D, lam, e = 1.0, 0.04, 1.0
    n, dt, rs, tol = (121, 0.2, (4, 6, 8, 10, 14), 1e-2) if dim == 2 else (61, 0.15, (6, 8, 10, 14, 18), 2.5e-2)
    g = oracle.Grid(dim, n, n, n if dim == 3 else 1, h=1.0, D=D, lam=lam, dt=dt)
    c = n // 2
    cell = c + n * c + (n * n * c if dim == 3 else 0)
    shape = (n,) * dim
    ell = np.sqrt(D / lam)
    none = (np.zeros((dim, 0)), np.zeros((dim, 0)), np.zeros(0, np.uint8))
    C, *_ = oracle.run(g, oracle.Cone(), np.zeros(shape), 0, int(12 / (lam * dt)), [cell], [e], None, *none)

    def along(axis, r):
        idx = [c] * dim
        idx[axis] += r
        return C[tuple(reversed(idx))]

    def green(r):
        if dim == 2:
            return e / dt / (2 * np.pi * D) * k0(r / ell)
        return e / dt / (4 * np.pi * D * r) * np.exp(-r / ell)

    errs = []
    for r in (3,) + rs:
        vals = [along(ax, r) for ax in range(dim)] + [along(0, -r)]
        np.testing.assert_allclose(vals, vals[0], rtol=1e-12)          # the same in every axis direction
        errs.append(abs(vals[0] / green(r) - 1.0))
    assert max(errs[1:]) <= tol, errs
    assert errs[0] > errs[1] > errs[3]                                 # O(h^2 / r^2) near the source
