"""Directed graphs: SCCs and the alpha/omega bounds of Section 2.3, and the
top-k / farness through Lemma 2's stopping rule, against the oracle."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1507_01490_gb300 import _build, bcm
    _build.build_cuda()
    bcm.load()
    return bcm


def directed_graphs(gen):
    ex = json.load(open(os.path.join(GOLDEN, "scc_dag_example.json")))
    a = np.array(ex["arcs"])
    gs = [gen.csr_from_arcs(ex["n"], a[:, 0], a[:, 1], directed=True, name="golden_scc"),
          gen.dpath(8), gen.dcycle(9), gen.empty(5, directed=True), gen.dpath(1),
          gen.disjoint_union(gen.dcycle(4), gen.dpath(3), gen.dcycle(4)),
          gen.relabel(gen.dcycle(15), seed=2),
          gen.with_self_loops_and_repeats(gen.gnp(40, 0.05, seed=7, directed=True), seed=3),
          gen.rmat(9, 6, seed=8), gen.rmat(11, 8, seed=3)]
    arcs = [(v, c) for v in range(31) for c in (2 * v + 1, 2 * v + 2) if c < 31]
    gs.append(gen.csr_from_arcs(31, [p for p, _ in arcs], [q for _, q in arcs], directed=True, name="outtree"))
    for s in range(8):
        gs.append(gen.gnp(50 + 29 * s, 0.012 + 0.01 * (s % 4), seed=200 + s, directed=True))
    return gs


def _partition(labels):
    groups = {}
    for v, c in enumerate(np.asarray(labels).tolist()):
        groups.setdefault(c, []).append(v)
    return sorted(tuple(x) for x in groups.values())


@pytest.mark.parametrize("refined", [True, False])
def test_scc_alpha_omega(B, gen, orc, refined):
    for g in directed_graphs(gen):
        ocomp, oal, oom, onc = orc.alpha_omega_refined(g) if refined else orc.alpha_omega(g)
        with B.BcmGraph.from_graph(g, flags=0 if refined else B.BCM_PLAIN_BOUNDS) as h:
            comp, al, om, nc = h.scc_bounds()
            order, lo, hi = h.preprocess()
        assert nc == onc, g.name
        assert _partition(comp) == _partition(ocomp), g.name
        firsts = {}
        for v, c in enumerate(comp.tolist()):
            firsts.setdefault(c, v)
        assert sorted(firsts, key=firsts.get) == list(range(nc)), g.name
        assert np.array_equal(al, oal) and np.array_equal(om, oom), g.name
        assert np.array_equal(lo, oal) and np.array_equal(hi, oom), g.name
        assert np.array_equal(order, orc.order(g)), g.name


@pytest.mark.parametrize("lanes", [64, 256])
def test_topk_and_farness_directed(B, gen, orc, lanes):
    for g in directed_graphs(gen):
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            gf, gr, _ = h.farness_all(grid_lanes=lanes)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), g.name
            gf, gr, _ = h.farness_all(lanes=lanes, flags=B.BCM_CTA_ONLY)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), g.name
            gf, gr, _ = h.farness_all(grid_lanes=lanes, flags=B.BCM_ALL_PULL)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), (g.name, "pull")
            for k in sorted({1, 2, 5, 10, 100, min(g.n, 1024), min(g.n + 3, 1024)} - {0}):
                exp = orc.topk(f, r, k)
                for flags, pd in ((0, 0), (B.BCM_CTA_ONLY, 0), (B.BCM_GRID_ONLY, 0), (B.BCM_GRID_ONLY | B.BCM_ALL_PULL, 0),
                                  (B.BCM_GRID_ONLY | B.BCM_NO_PULL, 0)):
                    ids, tf, tr, st = h.topk(k, lanes=lanes, grid_lanes=lanes, flags=flags, pull_div=pd)
                    assert np.array_equal(ids, exp), (g.name, k, flags)
                    assert np.array_equal(tf, f[exp]) and np.array_equal(tr, r[exp]), (g.name, k)


@pytest.mark.parametrize("refined", [True, False])
def test_plain_equals_oracle_bcm_directed(B, gen, orc, refined):
    for g in directed_graphs(gen):
        with B.BcmGraph.from_graph(g, flags=0 if refined else B.BCM_PLAIN_BOUNDS) as h:
            for k in (1, 4):
                ids, gf, gr, st = h.topk(k, flags=B.BCM_PLAIN)
                oi, of, orr, ost = orc.bcm(g, k, early_test=True, refined=refined)
                assert np.array_equal(ids, oi) and np.array_equal(gf, of), (g.name, k)
                assert st["m_vis"] == ost["m_vis"] and st["cut"] == ost["cut"], (g.name, k)


def test_rmat_scale14(B, gen, orc):
    g = gen.rmat(14, 16, seed=3)
    f, r = orc.farness_all(g)
    ocomp, oal, oom, onc = orc.alpha_omega_refined(g)
    with B.BcmGraph.from_graph(g) as h:
        comp, al, om, nc = h.scc_bounds()
        assert nc == onc and np.array_equal(al, oal) and np.array_equal(om, oom)
        for k in (1, 10, 100):
            for lanes in (64, 128, 256):
                ids, tf, tr, st = h.topk(k, lanes=lanes)
                exp = orc.topk(f, r, k)
                assert np.array_equal(ids, exp) and np.array_equal(tf, f[exp]) and np.array_equal(tr, r[exp])
