"""Per-lane level state of the BFS kernels (BCM_TRACE_LANES) against the
oracle, and the no-cut replay (BCM_NO_CUT).

At every level d a lane (one source v) holds Table 1's quantities: n_d (the
vertices within distance d), f_d (their distance sum) and gamma~_{d+1} (the
degree sum over Gamma_d, with the footnote's deg(u) - 1 for d >= 1 on
undirected graphs).  The records are checked:

* against BFS distances from scipy (a library routine independent of both
  the kernels and the oracle): n_d, f_d and gamma~_{d+1} exactly;
* against the oracle's Lemma 1 trace: f~_d(v, x) = f_d - gamma~_{d+1} +
  (d+2)(x - n_d) at x = r(v) (undirected) or at alpha(v) and omega(v)
  (directed, Lemma 2) equals oracle.bound_trace;
* gamma_{d+1} <= gamma~_{d+1} between consecutive records;
* a completed lane ends at its eccentricity with f(v) and r(v) of the
  oracle; a cut lane's bound at its last level ranks after the final k-th
  entry, so the cut was allowed by the threshold it could have read.

Each kernel is checked alone: per-CTA waves, grid-wide waves by push and by
pull, the plain one-source kernel, the one-source-per-CTA kernel (with and
without a grid-wide pass behind it), and the default schedule (seed wave,
prefilter, per-CTA waves).
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

pytestmark = pytest.mark.gpu


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


def _graphs(gen):
    return [gen.ba(400, 3, seed=31), gen.chung_lu(1 << 10, 6.0, 2.3, seed=32), gen.rmat(9, 8, seed=33),
            gen.grid_lcc(16, 20, 0.05, seed=34)]


def _dist(g):
    src = np.repeat(np.arange(g.n), g.degrees())
    a = sp.csr_matrix((np.ones(g.m), (src, g.col.astype(np.int64))), shape=(g.n, g.n))
    return shortest_path(a, method="D", directed=True, unweighted=True)


def _key(f, r):
    return (0, 1) if r <= 1 else ((r - 1) ** 2, f)


def _rank_before(a, b):
    (Na, Fa, ia), (Nb, Fb, ib) = a, b
    if Na * Fb != Nb * Fa:
        return Na * Fb > Nb * Fa
    return ia < ib


def _parse(recs):
    recs = np.asarray(recs, dtype=np.uint64)
    kind = (recs[:, 1] >> np.uint64(60)).astype(int)
    vid = ((recs[:, 1] >> np.uint64(32)) & np.uint64(0xfffffff)).astype(int)
    lvl = (recs[:, 1] & np.uint64(0xffffffff)).astype(int)
    a = recs[:, 2].astype(object)
    b = recs[:, 3].astype(object)
    levels = [(v, d, int(x), int(y) & 0xffffffff, int(y) >> 32)
              for k, v, d, x, y in zip(kind, vid, lvl, a, b) if k == 3]
    ends = [(v, d, int(x), int(y) & 0xffffffff, int(y) >> 32)
            for k, v, d, x, y in zip(kind, vid, lvl, a, b) if k == 4]
    return levels, ends


MODES = [("cta", dict(flags_extra="CTA_ONLY")), ("grid_push", dict(flags_extra="GRID_ONLY|NO_PULL")),
         ("grid_pull", dict(flags_extra="GRID_ONLY|ALL_PULL")), ("plain", dict(flags_extra="PLAIN")),
         ("default", dict(flags_extra="")), ("sparse", dict(flags_extra="SPARSE")),
         ("sparse_cta", dict(flags_extra="SPARSE|CTA_ONLY"))]


def _flags(B, names):
    f = 0
    for nm in filter(None, names.split("|")):
        f |= getattr(B, "BCM_" + nm)
    return f


@pytest.mark.parametrize("mode", [m[0] for m in MODES])
def test_lane_states_match_bfs_and_lemma1(B, gen, orc, mode):
    kw = dict(MODES)[mode]
    for g in _graphs(gen):
        dist = _dist(g)
        of, orr = orc.farness_all(g)
        deg = g.degrees()
        foot = 0 if g.directed else 1
        if g.directed:
            _, al, om, _ = orc.alpha_omega_refined(g)
        k = 5
        with B.BcmGraph.from_graph(g) as h:
            flags = B.BCM_TRACE | B.BCM_TRACE_LANES | _flags(B, kw["flags_extra"])
            ids, far, reach, st = h.topk(k, flags=flags, pull_div=kw.get("pull_div", 0))
            recs, cnt = h.trace()
        assert cnt <= len(recs), "trace truncated: use a smaller graph"
        exp_ids, exp_f, exp_r = orc.topk_exhaustive(g, k)
        assert np.array_equal(ids, exp_ids) and np.array_equal(far, exp_f) and np.array_equal(reach, exp_r)
        levels, ends = _parse(recs)
        assert levels and ends, (g.name, mode)
        per = {}
        for v, d, f, nd, gt in levels:
            dv = dist[v]
            fin = np.isfinite(dv)
            lv = dv[fin].astype(np.int64)
            within = lv <= d
            assert nd == int(within.sum()), (g.name, mode, v, d)
            assert f == int(lv[within].sum()), (g.name, mode, v, d)
            ring = np.nonzero(fin)[0][lv == d]
            exp_gt = int(deg[ring].sum()) - (foot * len(ring) if d >= 1 else 0)
            assert gt == exp_gt, (g.name, mode, v, d)
            xs = [int(orr[v])] if not g.directed else [int(al[v]), int(om[v])]
            for x in xs:
                tr = orc.bound_trace(g, v, x, orc.GT_FOOTNOTE if foot else orc.GT_TABLE1)
                assert d < len(tr) and f - gt + (d + 2) * (x - nd) == int(tr[d]), (g.name, mode, v, d, x)
            prev = per.setdefault(v, {}).get(d)
            assert prev is None or prev == (f, nd, gt), "a repeated run of a source gives other states"
            per[v][d] = (f, nd, gt)
        for v, st_v in per.items():
            for d, (f, nd, gt) in st_v.items():
                if d + 1 in st_v:
                    assert st_v[d + 1][1] - nd <= gt, "gamma_{d+1} > gamma~_{d+1}"
        kth = _key(int(far[-1]), int(reach[-1])) + (int(ids[-1]),)
        ended = set()
        for v, d, f, nd, cut in ends:
            ended.add(v)
            if not cut:
                assert f == int(of[v]) and nd == int(orr[v]), (g.name, mode, v)
                assert d == int(np.nanmax(np.where(np.isfinite(dist[v]), dist[v], np.nan))), (g.name, mode, v)
                continue
            gt = per[v][d][2]
            xs = [int(orr[v])] if not g.directed else [int(al[v]), int(om[v])]
            weak, strict = True, True
            for x in xs:
                ft = f - gt + (d + 2) * (x - nd)
                lhs, rhs = ft * kth[0], kth[1] * (x - 1) ** 2
                weak = weak and lhs >= rhs
                strict = strict and lhs > rhs
            assert strict or (weak and v > kth[2]), ("cut not allowed by the final k-th", g.name, mode, v, d)
        assert ended == set(range(g.n)), (g.name, mode, "sources without an end record")


@pytest.mark.parametrize("k", [1, 10])
def test_no_cut_replay_equals_exhaustive(B, gen, orc, k):
    """Without the bound every BFS runs to its end (Algorithm 1 is then the
    textbook algorithm); the top-k is the oracle's and the one bcm_farness_all's
    values rank to."""
    for g in _graphs(gen) + [gen.ba(2000, 3, seed=1)]:
        exp = orc.topk_exhaustive(g, k)
        with B.BcmGraph.from_graph(g) as h:
            ids, far, reach, st = h.topk(k, flags=B.BCM_NO_CUT)
            fa, ra, _ = h.farness_all()
        assert st["cut"] == 0 and st["completed"] >= g.n, (g.name, st["cut"], st["completed"])
        assert np.array_equal(ids, exp[0]) and np.array_equal(far, exp[1]) and np.array_equal(reach, exp[2])
        fids = orc.topk(fa, ra, k)
        assert np.array_equal(fids, ids) and np.array_equal(fa[fids], far) and np.array_equal(ra[fids], reach)
