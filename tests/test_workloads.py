"""The seeded synthetic workloads match their stated recipes (CPU only).

The five configurations of the benchmark (2D 128^2, 2D 2048^2, 3D 256^3, the
512-instance batch, the 1024^2 adjoint workload) and the connectivity workload
are drawn by paper_1405_3331_gb300/workloads.py; these checks pin the sizes,
physics and distributions stated for them, the explicit scheme's stability and
positivity (D dt / h^2 <= 1 / (2 dim), lambda dt + 2 dim D dt / h^2 <= 1), and
that a seed fixes every array.
"""
import numpy as np
import pytest

from paper_1405_3331_gb300 import workloads as W


def _stable(w):
    alpha = w.D * w.dt / (w.h * w.h)
    return alpha <= 1.0 / (2 * w.dim) + 1e-12 and w.lam * w.dt + 2 * w.dim * alpha <= 1.0 + 1e-12


@pytest.mark.parametrize("make,dim,shape,n_src,n_axons,nsteps,D,lam,dt", [
    (W.config_c1, 2, (128, 128), 4, 64, 500, 1.0, 0.01, 0.2),
    (W.config_c2, 2, (2048, 2048), 64, 16384, 5000, 1.0, 0.005, 0.2),
    (W.config_c3, 3, (256, 256, 256), 128, 65536, 2000, 1.0, 0.01, 0.15),
    (W.config_c5, 2, (1024, 1024), 32, 4096, 2000, 1.0, 0.01, 0.2),
])
def test_single_grid_configurations(make, dim, shape, n_src, n_axons, nsteps, D, lam, dt):
    w = make()
    assert (w.dim, w.shape, w.n_src, w.n_axons, w.nsteps) == (dim, shape, n_src, n_axons, nsteps)
    assert (w.D, w.lam, w.dt, w.h) == (D, lam, dt, 1.0)
    assert _stable(w)
    assert np.unique(w.src_cell).size == n_src and w.src_cell.min() >= 0 and w.src_cell.max() < w.n_cells
    hi = (np.array(shape[::-1], float) - 1.0)[:, None]
    assert np.all(w.pos >= 0.0) and np.all(w.pos <= hi)
    np.testing.assert_allclose(np.linalg.norm(w.dir.astype(np.float64), axis=0), 1.0, atol=1e-6)
    assert w.active.all()


def test_emissions_and_stop_radius():
    c1, c2 = W.config_c1(), W.config_c2()
    assert np.all(c1.src_emit == 1.0)
    assert c2.src_emit.min() >= 0.5 and c2.src_emit.max() <= 2.0 and np.unique(c2.src_emit).size > 1
    assert c2.stop_radius == 2.0
    # the 2048^2 cones start outside the stop radius of every source
    src = np.stack([c2.src_cell % c2.nx, c2.src_cell // c2.nx]).astype(np.float64)
    d2 = ((c2.pos[:, :, None].astype(np.float64) - src[:, None, :]) ** 2).sum(axis=0)
    assert d2.min() > c2.stop_radius ** 2


def test_adjoint_configuration_has_targets_clamp_and_a_zero_map():
    w = W.config_c5()
    assert w.wall_mode == 1 and w.stop_radius <= 0.0
    assert w.targets is not None and w.targets.shape == (2, w.n_axons)
    assert w.src_map is not None and not w.src_map.any()


def test_batch_distributions():
    ws = W.config_c4()
    assert len(ws) == 512
    nx = np.array([w.nx for w in ws]); ny = np.array([w.ny for w in ws])
    D = np.array([w.D for w in ws]); lam = np.array([w.lam for w in ws])
    assert nx.min() >= 64 and nx.max() <= 1024 and ny.min() >= 64 and ny.max() <= 1024
    assert D.min() >= 0.5 and D.max() <= 2.0
    assert lam.min() >= 1e-3 and lam.max() <= 1e-1
    np.testing.assert_allclose([w.dt * w.D for w in ws], 0.2)
    assert all(_stable(w) for w in ws)
    assert min(w.n_src for w in ws) >= 4 and max(w.n_src for w in ws) <= 64
    assert min(w.n_axons for w in ws) >= 256 and max(w.n_axons for w in ws) <= 4096
    assert all(w.nsteps == 1000 for w in ws)
    cells = sum(w.n_cells for w in ws)
    assert 146.0e6 < cells < 147.0e6                       # 146.4 M nodes
    assert 1.1e6 < sum(w.n_axons for w in ws) < 1.2e6       # 1.15 M cones


def test_seeds_fix_every_array():
    a, b = W.config_c2(seed=11), W.config_c2(seed=11)
    for f in ("src_cell", "src_emit", "pos", "dir"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.pos, W.config_c2(seed=12).pos)


def test_connectivity_workload():
    """262,144 neurons, 4 cones each within 48 of their neuron, 95% active; about 0.75
    connections per cone and neuron 0 reaching over 90% of the neurons (checked here with an
    independent k-d tree and scipy's BFS)."""
    spatial = pytest.importorskip("scipy.spatial")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.sparse import csr_matrix
    gw = W.config_graph()
    m, n = gw.n_neurons, gw.n_cones
    assert (m, n, gw.grid, gw.radius, gw.cell) == (262144, 1048576, (1024, 1024), 2.0, 2.0)
    np.testing.assert_array_equal(gw.owner, np.repeat(np.arange(m), 4))
    reach = np.linalg.norm(gw.pos.astype(np.float64) - gw.npos[:, gw.owner].astype(np.float64), axis=0)
    assert reach.max() <= 48.0 + 1e-3
    assert np.all(gw.pos >= 0.0) and np.all(gw.pos <= 2047.0)
    assert 0.94 < gw.active.mean() < 0.96
    tree = spatial.cKDTree(gw.npos.T.astype(np.float64))
    act = gw.active.astype(bool)
    hits = tree.query_ball_point(gw.pos.T[act].astype(np.float64), gw.radius * (1 - 1e-9))
    src = np.repeat(gw.owner[act], [len(h) for h in hits])
    dst = np.concatenate([np.asarray(h, dtype=np.int64) for h in hits])
    keep = src != dst
    assert 0.70 < keep.sum() / n < 0.80
    A = csr_matrix((np.ones(keep.sum()), (src[keep], dst[keep])), shape=(m, m))
    order = csgraph.breadth_first_order(A, gw.source, directed=True, return_predecessors=False)
    assert order.size > 0.9 * m


def test_clustered_workload_recipe():
    """2048^2 physics of the default workload; 16,384 cones in four 48 x 48 squares of 4,096,
    wall clamp, no source stop."""
    w = W.config_c2_clustered()
    c2 = W.config_c2()
    assert (w.nx, w.ny, w.D, w.lam, w.dt, w.n_src, w.n_axons) == (c2.nx, c2.ny, c2.D, c2.lam, c2.dt, 64, 16384)
    assert w.wall_mode == 1 and w.stop_radius == 0.0
    for q, (cx, cy) in enumerate([(512, 512), (1536, 512), (512, 1536), (1536, 1536)]):
        p = w.pos[:, q * 4096:(q + 1) * 4096]
        assert np.all(np.abs(p[0] - cx) <= 24) and np.all(np.abs(p[1] - cy) <= 24)
