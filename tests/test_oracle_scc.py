"""Pins the oracle's SCCs and Section 2.3's alpha/omega bounds."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _partition(labels):
    groups = {}
    for v, c in enumerate(np.asarray(labels).tolist()):
        groups.setdefault(c, []).append(v)
    return sorted(tuple(x) for x in groups.values())


def _scipy_scc(g):
    a = sp.csr_matrix((np.ones(g.m), g.col.astype(np.int64), g.row_ptr.astype(np.int64)),
                      shape=(g.n, g.n))
    return connected_components(a, directed=True, connection="strong")


def test_golden_example(orc, gen):
    ex = json.load(open(os.path.join(GOLDEN, "scc_dag_example.json")))
    a = np.array(ex["arcs"])
    g = gen.csr_from_arcs(ex["n"], a[:, 0], a[:, 1], directed=True)
    comp, al, om, nc = orc.alpha_omega(g)
    assert nc == len(ex["scc_sets"])
    assert _partition(comp) == sorted(tuple(s) for s in ex["scc_sets"])
    assert al.tolist() == ex["alpha"]
    assert om.tolist() == ex["omega"]
    f, r = orc.farness_all(g)
    assert r.tolist() == ex["reach"]


@pytest.mark.parametrize("seed,n,p", [(s, n, p) for s, (n, p) in enumerate(
    [(1, .5), (2, .6), (10, .1), (30, .05), (60, .03), (200, .008), (200, .02), (500, .003)] * 3)])
def test_scc_matches_scipy(orc, gen, seed, n, p):
    g = gen.gnp(n, p, seed=seed, directed=True)
    comp, nc = orc.scc(g)
    snc, slab = _scipy_scc(g)
    assert nc == snc
    assert _partition(comp) == _partition(slab)


def test_scc_rmat(orc, gen):
    g = gen.rmat(12, 8, seed=5)
    comp, nc = orc.scc(g)
    snc, slab = _scipy_scc(g)
    assert nc == snc and _partition(comp) == _partition(slab)


@pytest.mark.parametrize("seed,n,p", [(1, 40, .04), (2, 80, .02), (3, 150, .01), (4, 300, .006),
                                      (5, 60, .08), (6, 25, .15)])
def test_alpha_le_reach_le_omega(orc, gen, seed, n, p):
    g = gen.gnp(n, p, seed=seed, directed=True)
    comp, al, om, nc = orc.alpha_omega(g)
    f, r = orc.farness_all(g)
    assert (al <= r).all() and (r <= om).all() and (om <= n).all() and (al >= 1).all()
    # vertices of one SCC share their bounds and their reach
    for c in range(nc):
        vs = np.nonzero(comp == c)[0]
        assert len(set(r[vs].tolist())) == 1
        assert len(set(al[vs].tolist())) == 1 and len(set(om[vs].tolist())) == 1


def test_alpha_le_reach_le_omega_rmat(orc, gen):
    g = gen.rmat(11, 8, seed=7)
    comp, al, om, nc = orc.alpha_omega(g)
    f, r = orc.farness_all(g)
    assert (al <= r).all() and (r <= om).all()
    assert ((r == 1) == (al == 1)).all()      # alpha = 1 exactly for the vertices reaching nothing else


def test_out_tree_and_chain(orc, gen):
    # complete binary out-tree on 31 vertices: omega is the subtree size = r,
    # alpha is 1 + the longest downward path
    arcs = [(v, c) for v in range(31) for c in (2 * v + 1, 2 * v + 2) if c < 31]
    g = gen.csr_from_arcs(31, [a for a, _ in arcs], [b for _, b in arcs], directed=True)
    comp, al, om, nc = orc.alpha_omega(g)
    f, r = orc.farness_all(g)
    assert nc == 31
    assert (om == r).all()
    depth = np.floor(np.log2(np.arange(31) + 1)).astype(int)
    assert (al == 5 - depth).all()
    # a directed chain: alpha = omega = r
    g = gen.dpath(12)
    comp, al, om, nc = orc.alpha_omega(g)
    f, r = orc.farness_all(g)
    assert (al == r).all() and (om == r).all()


def test_strongly_connected(orc, gen):
    g = gen.dcycle(9)
    comp, al, om, nc = orc.alpha_omega(g)
    assert nc == 1 and (al == 9).all() and (om == 9).all()


def test_refined_golden_example(orc, gen):
    ex = json.load(open(os.path.join(GOLDEN, "scc_refined_example.json")))
    a = np.array(ex["arcs"])
    g = gen.csr_from_arcs(ex["n"], a[:, 0], a[:, 1], directed=True)
    comp, al, om, nc = orc.alpha_omega(g)
    assert al.tolist() == ex["alpha_plain"] and om.tolist() == ex["omega_plain"]
    comp, al, om, nc = orc.alpha_omega_refined(g)
    assert al.tolist() == ex["alpha_refined"] and om.tolist() == ex["omega_refined"]
    assert orc.farness_all(g)[1].tolist() == ex["reach"]
    # the first fixture: its largest SCC reaches everything, so the bounds become exact
    ex1 = json.load(open(os.path.join(GOLDEN, "scc_dag_example.json")))
    a1 = np.array(ex1["arcs"])
    g1 = gen.csr_from_arcs(ex1["n"], a1[:, 0], a1[:, 1], directed=True)
    comp, al, om, nc = orc.alpha_omega_refined(g1)
    assert al.tolist() == ex1["reach"] and om.tolist() == ex1["reach"]


@pytest.mark.parametrize("seed,n,p", [(1, 40, .04), (2, 80, .02), (3, 150, .01), (4, 300, .006),
                                      (5, 60, .08), (6, 25, .15), (7, 500, .004)])
def test_refined_bounds_valid_and_tighter(orc, gen, seed, n, p):
    g = gen.gnp(n, p, seed=seed, directed=True)
    _, al0, om0, _ = orc.alpha_omega(g)
    comp, al, om, nc = orc.alpha_omega_refined(g)
    f, r = orc.farness_all(g)
    assert (al <= r).all() and (r <= om).all()
    assert (al >= al0).all() and (om <= om0).all()
    # the largest SCC (smallest member on ties) is measured exactly
    sizes = np.bincount(comp, minlength=nc)
    best = max(range(nc), key=lambda c: (sizes[c], -int(np.nonzero(comp == c)[0].min())))
    vs = np.nonzero(comp == best)[0]
    assert (al[vs] == r[vs]).all() and (om[vs] == r[vs]).all()


def test_refined_rmat(orc, gen):
    g = gen.rmat(12, 8, seed=7)
    _, al0, om0, _ = orc.alpha_omega(g)
    comp, al, om, nc = orc.alpha_omega_refined(g)
    f, r = orc.farness_all(g)
    assert (al <= r).all() and (r <= om).all()
    assert (om < om0).sum() > 0.1 * g.n          # it tightens a good share of the graph
