"""Pins the oracle's BCM (Algorithm 1 + BFSCut) and Lemma 1/2 bounds.

* Correctness claim of Section 2 (Algorithm 1 returns the textbook top-k):
  BCM's (ids, farness, reach) equal the exhaustive top-k on many graphs, for
  every bound variant and both test schedules.
* Lemma 1: f~_d(v, r(v)) <= f(v) at every level; Lemma 2 on digraphs.
* Closed forms, worked by hand, for the bound along a path and for the arcs
  BCM scans on a star and a complete graph (these fix the (d+2) factor, the
  sign of the gamma~ term and the tie rule).
"""
from fractions import Fraction

import numpy as np
import pytest

MODES = [(0, True), (0, False), (1, True), (1, False), (2, True), (2, False)]


def _graphs(gen):
    gs = [gen.path(9), gen.star(12), gen.cycle(11), gen.complete(7), gen.grid(5, 6),
          gen.dpath(8), gen.dcycle(9), gen.empty(4),
          gen.disjoint_union(gen.cycle(5), gen.cycle(5), gen.empty(1), gen.cycle(5)),
          gen.relabel(gen.cycle(12), seed=3), gen.relabel(gen.grid(4, 4), seed=5),
          gen.ba(200, 2, seed=11), gen.grid_lcc(12, 12, 0.1, seed=2),
          gen.with_self_loops_and_repeats(gen.grid(4, 5), seed=1)]
    for s in range(12):
        gs.append(gen.gnp(60 + 7 * s, 0.02 + 0.01 * (s % 4), seed=100 + s, directed=False))
        gs.append(gen.gnp(50 + 9 * s, 0.015 + 0.01 * (s % 5), seed=200 + s, directed=True))
    gs.append(gen.rmat(9, 6, seed=8))
    gs.append(gen.chung_lu(800, 6.0, 2.3, seed=4))
    return gs


def test_bcm_equals_exhaustive(orc, gen):
    for g in _graphs(gen):
        f_all, r_all = orc.farness_all(g)
        for k in sorted({1, 2, 3, 10, g.n, g.n + 4}):
            ids = orc.topk(f_all, r_all, k)
            for mode, early in MODES:
                if mode == 1 and g.directed:
                    continue
                bi, bf, br, st = orc.bcm(g, k, gamma_mode=mode, early_test=early)
                assert bi.tolist() == ids.tolist(), (g.name, k, mode, early)
                assert (bf == f_all[ids]).all() and (br == r_all[ids]).all()
                assert st["completed"] + st["cut"] == g.n


def test_bcm_workload_ba2000(orc, gen):
    g = gen.workload("ba2000")
    f_all, r_all = orc.farness_all(g)
    for k in (1, 10, 100):
        ids = orc.topk(f_all, r_all, k)
        bi, bf, br, st = orc.bcm(g, k)
        assert bi.tolist() == ids.tolist() and (bf == f_all[ids]).all()
        # the cut prunes most of the textbook work (k = 100 is 5% of this graph)
        assert st["m_vis"] < (0.05 if k <= 10 else 0.5) * g.m * g.n


def test_early_test_scans_no_more(orc, gen):
    for g in _graphs(gen)[:20]:
        for mode in (0, 2):
            a = orc.bcm(g, 3, gamma_mode=mode, early_test=True)[3]["m_vis"]
            b = orc.bcm(g, 3, gamma_mode=mode, early_test=False)[3]["m_vis"]
            assert a <= b


def test_lemma1_every_level(orc, gen):
    for g in _graphs(gen):
        if g.directed:
            continue
        f, r = orc.farness_all(g)
        for v in range(0, g.n, max(1, g.n // 15)):
            for mode in (0, 1, 2):
                tr = orc.bound_trace(g, v, int(r[v]), mode)
                assert (tr <= int(f[v])).all(), (g.name, v, mode)
            # at the last level the ball is all of R(v): f~ = f - gamma~ exactly
            last = orc.bound_trace(g, v, int(r[v]), 0)[-1]
            assert last <= int(f[v])


def test_lemma2_digraphs(orc, gen):
    for s in range(10):
        g = gen.gnp(70, 0.03, seed=300 + s, directed=True)
        comp, al, om, nc = orc.alpha_omega(g)
        f, r = orc.farness_all(g)
        for v in range(g.n):
            if r[v] <= 1:
                continue
            inv_c = Fraction(int(f[v]), (int(r[v]) - 1) ** 2)
            ta = orc.bound_trace(g, v, int(al[v]), 0)
            to = orc.bound_trace(g, v, int(om[v]), 0)
            for d in range(len(ta)):
                lam = min(Fraction(int(ta[d]), (int(al[v]) - 1) ** 2),
                          Fraction(int(to[d]), (int(om[v]) - 1) ** 2))
                assert lam <= inv_c, (s, v, d)


@pytest.mark.parametrize("n", [3, 6, 20])
def test_bound_along_path_closed_form(orc, gen, n):
    # vertex 0 of the path: Gamma_d = {d}, n_d = d+1, f_d = d(d+1)/2,
    # gamma~_{d+1} = deg(d): 1 at d = 0, 2 inside, 1 at the far end.
    g = gen.path(n)
    tr = orc.bound_trace(g, 0, n, 0)
    tr1 = orc.bound_trace(g, 0, n, 1)
    assert len(tr) == n
    for d in range(n):
        deg = 1 if d in (0, n - 1) else 2
        base = d * (d + 1) // 2 + (d + 2) * (n - d - 1)
        assert tr[d] == base - deg
        assert tr1[d] == base - (deg if d == 0 else deg - 1)


@pytest.mark.parametrize("n", [3, 5, 30])
def test_star_leaf_bound_is_tight(orc, gen, n):
    g = gen.star(n)
    assert orc.bound_trace(g, 1, n, 0)[0] == 2 * n - 3 == orc.farness_all(g)[0][1]


@pytest.mark.parametrize("n", [3, 8, 25])
def test_arcs_scanned_star(orc, gen, n):
    g = gen.star(n)
    # centre first (full BFS: 2(n-1) arcs), every leaf is then stopped at level 0:
    # before scanning its arc (early test) or after (Algorithm 2's schedule)
    st = orc.bcm(g, 1, early_test=True)[3]
    assert st["m_vis"] == 2 * (n - 1) and st["completed"] == 1 and st["cut"] == n - 1
    st = orc.bcm(g, 1, early_test=False)[3]
    assert st["m_vis"] == 3 * (n - 1)


@pytest.mark.parametrize("n", [3, 6, 12])
def test_arcs_scanned_complete_ties(orc, gen, n):
    g = gen.complete(n)
    # all vertices tie; vertex 0 completes, every later one meets the tie at
    # level 0 (f~_0 = n-1 = f_k) and loses it on its larger id
    ids, f, r, st = orc.bcm(g, 1, early_test=True)
    assert ids.tolist() == [0] and st["m_vis"] == n * (n - 1) and st["cut"] == n - 1
    st = orc.bcm(g, 1, early_test=False)[3]
    assert st["m_vis"] == n * (n - 1) + (n - 1) ** 2
    ids, f, r, st = orc.bcm(g, 2, early_test=True)
    assert ids.tolist() == [0, 1] and st["m_vis"] == 2 * n * (n - 1)


def test_bcm_refined_bounds_equal_exhaustive(orc, gen):
    for s in range(8):
        g = gen.gnp(60 + 20 * s, 0.02 + 0.005 * (s % 3), seed=400 + s, directed=True)
        f_all, r_all = orc.farness_all(g)
        for k in (1, 3, 10):
            ids = orc.topk(f_all, r_all, k)
            for early in (True, False):
                bi, bf, br, st = orc.bcm(g, k, early_test=early, refined=True)
                assert bi.tolist() == ids.tolist()
    g = gen.rmat(11, 8, seed=3)
    f_all, r_all = orc.farness_all(g)
    ids = orc.topk(f_all, r_all, 10)
    a = orc.bcm(g, 10, refined=False)
    b = orc.bcm(g, 10, refined=True)
    assert a[0].tolist() == ids.tolist() == b[0].tolist()
    assert b[3]["m_vis"] <= a[3]["m_vis"]


def _bounds(orc, g):
    if g.directed:
        _, al, om, _ = orc.alpha_omega(g)
        return al, om
    _, r = orc.farness_all(g)
    return r, r


def _shard(n, index, count, chunk=64):
    p = np.arange(n)
    return p[(p // chunk) % count == index]


def _key(f, r, v):
    return (1, 0, 1, int(v)) if r <= 1 or f == 0 else (1, (int(r) - 1) ** 2, int(f), int(v))


def test_shard_runner_whole_order_is_bcm(orc, gen):
    """One shard holding every source, with no outside key, is Algorithm 1
    itself, whether run at once or a few sources at a time."""
    for g in _graphs(gen)[::3]:
        order = orc.order(g)
        for k in (1, 3, 10):
            ids, f, r, st = orc.bcm(g, k)
            for step in (g.n + 1, 7):
                run = orc.ShardRun(g, k, order, _bounds(orc, g))
                while not run.step(step):
                    pass
                gi, gf, gr, gst = run.result()
                assert np.array_equal(gi, ids) and np.array_equal(gf, f) and np.array_equal(gr, r), (g.name, k)
                assert gst["m_vis"] == st["m_vis"] and gst["cut"] == st["cut"], (g.name, k, step)


@pytest.mark.parametrize("count", [2, 3])
def test_shard_runner_with_the_global_kth_key(orc, gen, count):
    """Offered the graph's exact k-th key, each shard still returns every
    top-k member it holds, the merged lists are the textbook top-k, and no
    shard scans more arcs than without the key (a stronger threshold can only
    stop sources earlier)."""
    with_key = without = 0
    for g in _graphs(gen)[::2]:
        f_all, r_all = orc.farness_all(g)
        order = orc.order(g)
        for k in (1, 5, 10):
            exp = orc.topk(f_all, r_all, k)
            if len(exp) < k:
                continue
            kth = _key(f_all[exp[-1]], r_all[exp[-1]], exp[-1])
            lists = []
            for s in range(count):
                src = order[_shard(g.n, s, count)]
                base = orc.ShardRun(g, k, src, _bounds(orc, g))
                base.step(len(src) + 1)
                run = orc.ShardRun(g, k, src, _bounds(orc, g))
                run.offer(kth)
                run.step(len(src) + 1)
                ids, f, r, st = run.result()
                assert set(exp.tolist()) & set(src.tolist()) <= set(ids.tolist()), (g.name, k, s)
                assert st["m_vis"] <= base.result()[3]["m_vis"], (g.name, k, s)
                with_key += st["m_vis"]
                without += base.result()[3]["m_vis"]
                lists.append(ids)
            # the merge: the best k of the union (sorted by id, since the oracle's
            # top-k breaks ties by array position)
            cat = np.sort(np.concatenate(lists)).astype(np.uint32)
            assert np.array_equal(cat[orc.topk(f_all[cat], r_all[cat], k)], exp), (g.name, k)
    assert with_key < without
