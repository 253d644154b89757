"""The connectivity stage on the GPU (include/cue_graph.h) against the FP64 oracle: integer
results, so every comparison is exact (the edge list of cue_connect is compared as a set,
its order being unspecified)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_1405_3331_gb300 import build
    build.build()
    from paper_1405_3331_gb300 import graph
    return graph


def _t(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


@pytest.mark.parametrize("dim,n,grid,cell", [(2, 0, [4, 3], 1.0), (2, 5, [10, 1], 1.0), (2, 20000, [64, 48], 1.3),
                                             (3, 30000, [20, 17, 9], 2.1), (2, 7, [1, 1], 5.0)])
def test_binning_matches_oracle(g, dim, n, grid, cell):
    import torch
    rng = np.random.default_rng(n + dim)
    ext = np.array(grid[:dim])[:, None] * cell
    pos = (rng.uniform(-0.05, 1.05, (dim, n)) * ext).astype(np.float32)   # a few outside: clamped
    got = [t.cpu().numpy() for t in g.bin_points(_t(pos, torch.float32), cell, grid)]
    want = oracle.bin_points(pos.astype(np.float64), np.float32(cell), grid)
    for x, y, what in zip(got, want, ("cell_of", "sorted_id", "cell_start", "cell_end")):
        np.testing.assert_array_equal(x, y, err_msg=what)


@pytest.mark.parametrize("dim", [2, 3])
def test_connections_match_oracle(g, dim):
    import torch
    rng = np.random.default_rng(7 + dim)
    n, m, r = 20000, 3000, 1.5
    grid = [40, 30, 12][:dim]
    cell = 1.5
    ext = np.array(grid)[:, None] * cell
    npos = (rng.uniform(0, 1, (dim, m)) * ext).astype(np.float32)
    pos = (rng.uniform(0, 1, (dim, n)) * ext).astype(np.float32)
    owner = rng.integers(0, m, n).astype(np.int32)
    active = (rng.uniform(size=n) < 0.8).astype(np.uint8)
    binned = g.bin_points(_t(npos, torch.float32), cell, grid)
    src, dst, cnt = g.connect(_t(pos, torch.float32), _t(owner, torch.int32), _t(active, torch.uint8),
                              _t(npos, torch.float32), r, cell, grid, binned, cap=200000)
    k = int(cnt.item())
    got = sorted(zip(src[:k].cpu().numpy().tolist(), dst[:k].cpu().numpy().tolist()))
    ws, wd = oracle.connect(pos.astype(np.float64), owner, active, npos.astype(np.float64), np.float32(r))
    assert k == ws.size > 0
    assert got == sorted(zip(ws.tolist(), wd.tolist()))
    # a cap below the count: the count is still the full count, only cap pairs are written
    src2, dst2, cnt2 = g.connect(_t(pos, torch.float32), _t(owner, torch.int32), _t(active, torch.uint8),
                                 _t(npos, torch.float32), r, cell, grid, binned, cap=10)
    assert int(cnt2.item()) == k


def test_adjacency_list_matches_oracle(g):
    import torch
    rng = np.random.default_rng(17)
    nv, ne = 5000, 60000
    src = rng.integers(0, nv, ne).astype(np.int32)
    dst = rng.integers(0, nv, ne).astype(np.int32)
    src[:50] = -1                                          # skipped
    row, col, m = g.csr(nv, _t(src, torch.int32), _t(dst, torch.int32), _t([ne - 100], torch.int32))
    keep = np.arange(ne) < ne - 100
    keep &= src >= 0
    wr, wc = oracle.csr(nv, src[keep], dst[keep])
    np.testing.assert_array_equal(row.cpu().numpy(), wr)
    assert int(m.item()) == wc.size
    np.testing.assert_array_equal(col.cpu().numpy()[: wc.size], wc)


@pytest.mark.parametrize("shape", ["random", "path", "star", "empty"])
def test_bfs_matches_oracle(g, shape):
    import torch
    rng = np.random.default_rng(23)
    if shape == "random":
        nv, ne = 20000, 60000
        src, dst = rng.integers(0, nv, ne), rng.integers(0, nv, ne)
    elif shape == "path":                                  # 5,000 levels: 5,001 barriers in one launch
        nv = 5000
        src, dst = np.arange(nv - 1), np.arange(1, nv)
    elif shape == "star":
        nv = 3000
        src, dst = np.zeros(nv - 1, int), np.arange(1, nv)
    else:
        nv = 100
        src, dst = np.zeros(0, int), np.zeros(0, int)
    wr, wc = oracle.csr(nv, src, dst)
    for s in (0, int(rng.integers(nv))):
        lev = g.bfs(_t(wr, torch.int32), _t(wc if wc.size else np.zeros(1), torch.int32), s).cpu().numpy()
        np.testing.assert_array_equal(lev, oracle.bfs(wr, wc, s))


def test_pipeline_from_a_simulation(g):
    """Cones grown by the simulation connect to neurons; the connection graph's BFS levels."""
    import torch
    from paper_1405_3331_gb300 import cue
    from paper_1405_3331_gb300 import workloads as W
    w = W.make("net", 2, 256, 256, n_src=16, n_axons=4000, C0="smooth", seed=90, wall_mode=1)
    sim = cue.Simulation(w)
    sim.sim_run(200)
    sim.check()
    _, pos, _, act, _, _ = sim.snapshot()
    sim.close()
    rng = np.random.default_rng(91)
    m = 800
    npos = rng.uniform(0, 255, (2, m)).astype(np.float32)
    owner = (np.arange(w.n_axons) % m).astype(np.int32)
    grid, cell, r = [128, 128], 2.0, 2.0
    binned = g.bin_points(_t(npos, torch.float32), cell, grid)
    src, dst, cnt = g.connect(_t(pos, torch.float32), _t(owner, torch.int32), _t(act, torch.uint8),
                              _t(npos, torch.float32), r, cell, grid, binned, cap=100000)
    row, col, mm = g.csr(m, src, dst, cnt)
    lev = g.bfs(row, col, 0).cpu().numpy()
    ws, wd = oracle.connect(pos.astype(np.float64), owner, act, npos.astype(np.float64), r)
    wr, wc = oracle.csr(m, ws, wd)
    np.testing.assert_array_equal(row.cpu().numpy(), wr)
    np.testing.assert_array_equal(col.cpu().numpy()[: wc.size], wc)
    np.testing.assert_array_equal(lev, oracle.bfs(wr, wc, 0))
    assert wc.size > 100 and (lev > 1).any()


def test_connectivity_at_the_benchmark_size(g):
    """The bench's connectivity workload (262,144 neurons, 1,048,576 cones): binning of every
    neuron against the oracle; the connections of the cones of the first 1,000 neurons against
    the oracle's brute-force pair test (as a set); the adjacency list and BFS levels of the whole
    graph by properties that hold at any size (rows sorted and distinct and covering exactly the
    distinct connections; every level one more than some predecessor's, no edge skipping one)."""
    import torch
    from paper_1405_3331_gb300 import workloads as W
    gw = W.config_graph()
    m, n = gw.n_neurons, gw.n_cones
    binned = g.bin_points(_t(gw.npos, torch.float32), gw.cell, gw.grid)
    want = oracle.bin_points(gw.npos.astype(np.float64), np.float32(gw.cell), gw.grid)
    for x, y, what in zip(binned, want, ("cell_of", "sorted_id", "cell_start", "cell_end")):
        np.testing.assert_array_equal(x.cpu().numpy(), y, err_msg=what)
    src, dst, cnt = g.connect(_t(gw.pos, torch.float32), _t(gw.owner, torch.int32), _t(gw.active, torch.uint8),
                              _t(gw.npos, torch.float32), gw.radius, gw.cell, gw.grid, binned, cap=4 * n)
    k = int(cnt.item())
    assert 0.5 * n < k < 1.2 * n, k
    s, d = src.cpu().numpy()[:k], dst.cpu().numpy()[:k]
    first = 1000
    cones = np.flatnonzero(gw.owner < first)
    ws_, wd_ = oracle.connect(gw.pos[:, cones].astype(np.float64), gw.owner[cones], gw.active[cones],
                              gw.npos.astype(np.float64), gw.radius, cap=16 * cones.size)
    sel = s < first
    assert sorted(zip(s[sel].tolist(), d[sel].tolist())) == sorted(zip(ws_.tolist(), wd_.tolist()))
    row, col, mm = g.csr(m, src, dst, cnt)
    row, e = row.cpu().numpy(), int(mm.item())
    col = col.cpu().numpy()[:e]
    assert row[0] == 0 and row[-1] == e and np.all(np.diff(row) >= 0)
    u = np.repeat(np.arange(m), np.diff(row))
    assert np.all((u[1:] != u[:-1]) | (col[1:] > col[:-1]))          # each row ascending, distinct
    pairs = np.unique(s.astype(np.int64) * m + d)
    np.testing.assert_array_equal(np.sort(u.astype(np.int64) * m + col), pairs)
    lev = g.bfs(_t(row, torch.int32), _t(col, torch.int32), gw.source).cpu().numpy()
    assert lev[gw.source] == 0 and (lev >= 0).sum() > m // 2
    lu, lv = lev[u], lev[col]
    reach = lu >= 0
    assert np.all(lv[reach] >= 0) and np.all(lv[reach] <= lu[reach] + 1)   # no edge skips a level
    best = np.full(m, np.iinfo(np.int64).max)
    np.minimum.at(best, col[reach], lu[reach].astype(np.int64) + 1)
    hit = lev > 0
    np.testing.assert_array_equal(best[hit], lev[hit])                      # each level from a predecessor
    assert np.all(lev[lev < 0] == -1) and not np.any((lev < 0) & (best < np.iinfo(np.int64).max))
