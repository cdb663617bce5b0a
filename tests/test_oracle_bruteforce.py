"""Pins the oracle against brute force and library routines.

* Floyd-Warshall all-pairs distances on graphs with n <= 10 (every undirected
  graph on 5 vertices, random digraphs on up to 10).
* scipy.sparse.csgraph's unweighted shortest paths on larger random graphs.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

INF = 10**9


def _floyd_warshall(n, arcs):
    d = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(d, 0)
    for u, w in arcs:
        if u != w:
            d[u, w] = 1
    for k in range(n):
        d = np.minimum(d, d[:, [k]] + d[[k], :])
    return d


def _fr_from_dist(d):
    reach = (d < INF).sum(axis=1)
    far = np.where(d < INF, d, 0).sum(axis=1)
    return far, reach


def _arcs(g):
    src = np.repeat(np.arange(g.n), g.degrees())
    return list(zip(src.tolist(), g.col.tolist()))


def test_all_undirected_graphs_on_5_vertices(orc, gen):
    n = 5
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        es = [p for i, p in enumerate(pairs) if mask >> i & 1]
        g = gen.csr_from_arcs(n, [a for a, _ in es], [b for _, b in es], directed=False)
        f, r = orc.farness_all(g, threads=1)
        ef, er = _fr_from_dist(_floyd_warshall(n, _arcs(g)))
        assert (f == ef).all() and (r == er).all(), es


@pytest.mark.parametrize("seed", range(40))
def test_random_digraphs_up_to_10(orc, gen, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 11))
    p = float(rng.uniform(0.05, 0.5))
    g = gen.gnp(n, p, seed=seed, directed=True)
    f, r = orc.farness_all(g, threads=1)
    ef, er = _fr_from_dist(_floyd_warshall(n, _arcs(g)))
    assert (f == ef).all() and (r == er).all()


@pytest.mark.parametrize("seed,directed,n,p", [
    (1, False, 300, 0.01), (2, True, 300, 0.01), (3, False, 200, 0.003),
    (4, True, 250, 0.006), (5, True, 120, 0.05)])
def test_scipy_shortest_paths(orc, gen, seed, directed, n, p):
    g = gen.gnp(n, p, seed=seed, directed=directed)
    a = sp.csr_matrix((np.ones(g.m), g.col.astype(np.int64), g.row_ptr.astype(np.int64)),
                      shape=(n, n))
    d = shortest_path(a, directed=True, unweighted=True)
    fin = np.isfinite(d)
    ef = np.where(fin, d, 0).sum(axis=1).astype(np.int64)
    er = fin.sum(axis=1)
    f, r = orc.farness_all(g)
    assert (f.astype(np.int64) == ef).all() and (r == er).all()


def test_workload_recipes_small_scale(orc, gen):
    """The named recipes at small sizes, against scipy."""
    for g in [gen.ba(300, 3, seed=1), gen.chung_lu(2000, 10.0, 2.3, seed=2),
              gen.rmat(10, 16, seed=3), gen.grid_lcc(30, 30, 0.05, seed=4)]:
        a = sp.csr_matrix((np.ones(g.m), g.col.astype(np.int64), g.row_ptr.astype(np.int64)),
                          shape=(g.n, g.n))
        src = np.arange(0, g.n, max(1, g.n // 97))
        d = shortest_path(a, directed=True, unweighted=True, indices=src)
        fin = np.isfinite(d)
        f, r = orc.farness_all(g, sources=src)
        assert (f.astype(np.int64) == np.where(fin, d, 0).sum(axis=1)).all(), g.name
        assert (r == fin.sum(axis=1)).all(), g.name


def test_threads_share_short_lists(orc, gen):
    """The exhaustive oracle hands out sources in grabs small enough that
    every thread takes work on a 64-source call, and the result does not
    depend on how many threads ran (each BFS is independent)."""
    g = gen.ba(3000, 3, seed=12)
    src = gen.uniform_u32(21, 64, g.n)
    f1, r1 = orc.farness_all(g, sources=src, threads=1)
    for t in (4, 16):
        info = {}
        f, r = orc.farness_all(g, sources=src, threads=t, info=info)
        assert info["threads_used"] == t
        assert np.array_equal(f, f1) and np.array_equal(r, r1)
    info = {}
    orc.farness_all(g, sources=src[:0], threads=8, info=info)
    assert info["threads_used"] == 0
