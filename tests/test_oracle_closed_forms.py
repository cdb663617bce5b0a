"""Pins the oracle's farness/reach (Table 1 definitions) to closed forms.

f(v) = sum of d(v, w) over R(v), r(v) = |R(v)|, both written out by hand for
families whose distances are known exactly.
"""
import numpy as np
import pytest


def _fr(orc, g):
    f, r = orc.farness_all(g, threads=2)
    return f.astype(np.int64), r.astype(np.int64)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 50])
def test_path(orc, gen, n):
    f, r = _fr(orc, gen.path(n))
    i = np.arange(n)
    assert (r == n).all()
    assert (f == i * (i + 1) // 2 + (n - 1 - i) * (n - i) // 2).all()


@pytest.mark.parametrize("n", [2, 3, 9, 40])
def test_star(orc, gen, n):
    f, r = _fr(orc, gen.star(n))
    assert f[0] == n - 1
    assert (f[1:] == 2 * n - 3).all()
    assert (r == n).all()


@pytest.mark.parametrize("n", [3, 4, 5, 10, 31])
def test_cycle(orc, gen, n):
    f, r = _fr(orc, gen.cycle(n))
    assert (f == n * n // 4).all() and (r == n).all()


@pytest.mark.parametrize("n", [1, 2, 6, 25])
def test_complete(orc, gen, n):
    f, r = _fr(orc, gen.complete(n))
    assert (f == n - 1).all() and (r == n).all()


@pytest.mark.parametrize("a,b", [(1, 1), (1, 5), (3, 4), (7, 7), (10, 3)])
def test_grid(orc, gen, a, b):
    f, r = _fr(orc, gen.grid(a, b))
    i, j = np.divmod(np.arange(a * b), b)
    rows = i * (i + 1) // 2 + (a - 1 - i) * (a - i) // 2
    cols = j * (j + 1) // 2 + (b - 1 - j) * (b - j) // 2
    assert (f == b * rows + a * cols).all()
    assert (r == a * b).all()


@pytest.mark.parametrize("n", [1, 2, 5, 33])
def test_directed_path(orc, gen, n):
    f, r = _fr(orc, gen.dpath(n))
    i = np.arange(n)
    assert (r == n - i).all()
    assert (f == (n - 1 - i) * (n - i) // 2).all()


@pytest.mark.parametrize("n", [2, 3, 8, 21])
def test_directed_cycle(orc, gen, n):
    f, r = _fr(orc, gen.dcycle(n))
    assert (r == n).all() and (f == n * (n - 1) // 2).all()


def test_disjoint_union(orc, gen):
    g = gen.disjoint_union(gen.path(4), gen.star(5), gen.complete(3), gen.empty(2))
    f, r = _fr(orc, g)
    assert r.tolist() == [4] * 4 + [5] * 5 + [3] * 3 + [1] * 2
    assert f.tolist() == [6, 4, 4, 6] + [4, 7, 7, 7, 7] + [2, 2, 2] + [0, 0]


def test_empty_graph(orc, gen):
    f, r = _fr(orc, gen.empty(5))
    assert (f == 0).all() and (r == 1).all()
    f, r = orc.farness_all(gen.empty(0))
    assert f.size == 0 and r.size == 0


def test_self_loops_and_repeats_change_nothing(orc, gen):
    for base in [gen.grid(4, 6), gen.gnp(40, 0.08, seed=3, directed=True)]:
        noisy = gen.with_self_loops_and_repeats(base, seed=9, frac=0.5)
        assert noisy.m > base.m
        f0, r0 = _fr(orc, base)
        f1, r1 = _fr(orc, noisy)
        assert (f0 == f1).all() and (r0 == r1).all()


def test_sources_subset_and_arc_counts(orc, gen):
    g = gen.grid(5, 5)
    f, r, a = orc.farness_all(g, sources=[24, 0, 12], arcs=True)
    fa, ra = orc.farness_all(g)
    assert f.tolist() == [fa[24], fa[0], fa[12]]
    # every vertex reaches the whole grid, so each BFS scans all m arcs
    assert (a == g.m).all()
