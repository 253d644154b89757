"""Pins of the oracle's connectivity stage (CPU only): uniform-grid binning by hash, sort and
cell start (Sec. 3.5, Table 1), the squared-distance connection test (Sec. 3.3), the adjacency
list (Sec. 3.4, Fig. 4) and breadth-first levels (Sec. 3.4, Fig. 5), against the paper's
worked example and against library definitions (numpy, scipy.sparse, networkx)."""
import os

import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_hash_sort.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        key, *pairs = line.split()
        rows[key] = [tuple(int(v) for v in p.split(":")) for p in pairs]
    return rows


def test_table1_example():
    g = _golden()
    cells = np.array([c for _, c in sorted(g["unsorted"])], np.float64)
    pos = np.stack([cells + 0.5, np.zeros_like(cells)])           # cell k holds x in [k, k+1)
    cell_of, sid, start, end = oracle.bin_points(pos, 1.0, [10, 1])
    assert [(int(cell_of[i]), int(i)) for i in sid] == g["sorted"]
    for c, s in g["start"]:
        assert start[c] == s
    for c, e in g["end"]:
        assert end[c] == e
    occupied = {c for c, _ in g["start"]}
    assert all(start[c] == -1 and end[c] == -1 for c in range(10) if c not in occupied)


@pytest.mark.parametrize("dim", [2, 3])
def test_binning_is_a_stable_sort_by_cell(dim):
    rng = np.random.default_rng(11 + dim)
    n = 5000
    grid = [17, 13, 7][:dim]
    pos = rng.uniform(-1.0, 25.0, (dim, n))                          # some points outside: clamped
    cell_of, sid, start, end = oracle.bin_points(pos, 1.5, grid)
    k = np.clip(np.floor(pos / 1.5).astype(np.int64), 0, np.array(grid)[:, None] - 1)
    lin = k[0] + grid[0] * (k[1] + (grid[1] * k[2] if dim == 3 else 0))
    np.testing.assert_array_equal(cell_of, lin)
    np.testing.assert_array_equal(sid, np.lexsort((np.arange(n), lin)))
    counts = np.bincount(lin, minlength=int(np.prod(grid)))
    occ = counts > 0
    np.testing.assert_array_equal(end[occ] - start[occ], counts[occ])
    np.testing.assert_array_equal(start[occ], np.cumsum(counts)[occ] - counts[occ])
    assert np.all(start[~occ] == -1) and np.all(end[~occ] == -1)


@pytest.mark.parametrize("dim", [2, 3])
def test_connections_are_the_pairs_within_the_radius(dim):
    rng = np.random.default_rng(21 + dim)
    n, m, r = 700, 300, 1.7
    pos = rng.uniform(0, 30, (dim, n))
    npos = rng.uniform(0, 30, (dim, m))
    owner = rng.integers(0, m, n).astype(np.int32)
    active = (rng.uniform(size=n) < 0.9).astype(np.uint8)
    src, dst = oracle.connect(pos, owner, active, npos, r)
    d2 = ((pos[:, :, None] - npos[:, None, :]) ** 2).sum(0)
    a, j = np.nonzero((d2 < r * r) & active.astype(bool)[:, None] & (owner[:, None] != np.arange(m)[None, :]))
    np.testing.assert_array_equal(src, owner[a])
    np.testing.assert_array_equal(dst, j)
    # the test is strict: a pair at exactly the radius does not connect
    s2, d2_ = oracle.connect(np.array([[0.0], [0.0]]), [0], None, np.array([[0.0, 3.0], [0.0, 4.0]]), 5.0)
    assert s2.size == 0


def test_adjacency_list_is_the_csr_of_the_distinct_edges():
    rng = np.random.default_rng(31)
    nv, ne = 400, 3000
    src = rng.integers(0, nv, ne).astype(np.int32)
    dst = rng.integers(0, nv, ne).astype(np.int32)
    row, col = oracle.csr(nv, src, dst)
    A = sp.coo_matrix((np.ones(ne), (src, dst)), shape=(nv, nv)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    np.testing.assert_array_equal(row, A.indptr)
    np.testing.assert_array_equal(col, A.indices)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bfs_levels_are_shortest_hop_counts(seed):
    rng = np.random.default_rng(41 + seed)
    nv = 600
    G = nx.gnm_random_graph(nv, 900, seed=seed, directed=True)
    src = np.array([u for u, v in G.edges()], np.int32)
    dst = np.array([v for u, v in G.edges()], np.int32)
    row, col = oracle.csr(nv, src, dst)
    s = int(rng.integers(nv))
    lev = oracle.bfs(row, col, s)
    want = nx.single_source_shortest_path_length(G, s)
    for v in range(nv):
        assert lev[v] == want.get(v, -1)


def test_bfs_on_a_path_and_without_edges():
    nv = 50
    row, col = oracle.csr(nv, np.arange(nv - 1), np.arange(1, nv))
    np.testing.assert_array_equal(oracle.bfs(row, col, 0), np.arange(nv))
    np.testing.assert_array_equal(oracle.bfs(row, col, 10), np.r_[-np.ones(10), np.arange(nv - 10)])
    row0, col0 = oracle.csr(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    np.testing.assert_array_equal(oracle.bfs(row0, col0, 2), [-1, -1, 0, -1, -1])
