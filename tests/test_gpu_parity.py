"""CUDA path vs the oracle, element by element, through the C-ABI.

Integer outputs, so the bar is bit-exact: top-k ids, farness and reach; the
farness/reach of every vertex; the processing order; r(v) or alpha/omega.
Sizes here are ones the oracle finishes in seconds; full-size workloads are
in test_gpu_fullsize.py.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LANES = [64, 128, 256]


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


def undirected_graphs(gen):
    gs = [gen.path(9), gen.star(12), gen.cycle(11), gen.complete(7), gen.grid(5, 6), gen.empty(4),
          gen.path(1), gen.path(2),
          gen.disjoint_union(gen.cycle(5), gen.cycle(5), gen.empty(1), gen.cycle(5)),
          gen.relabel(gen.cycle(12), seed=3), gen.relabel(gen.grid(4, 4), seed=5),
          gen.ba(200, 2, seed=11), gen.grid_lcc(12, 12, 0.1, seed=2),
          gen.with_self_loops_and_repeats(gen.grid(4, 5), seed=1),
          gen.star(300), gen.grid(17, 19),
          # in-hubs (more than 128 in-arcs) scanned in pieces by pulled levels: every vertex of
          # K_260, a centre with 4 pieces, the hubs of a denser BA graph
          gen.complete(260), gen.star(1000), gen.ba(3000, 8, seed=12)]
    for s in range(6):
        gs.append(gen.gnp(60 + 37 * s, 0.02 + 0.01 * (s % 4), seed=100 + s, directed=False))
    gs.append(gen.chung_lu(3000, 6.0, 2.3, seed=4))
    return gs


def _partition(labels):
    groups = {}
    for v, c in enumerate(np.asarray(labels).tolist()):
        groups.setdefault(c, []).append(v)
    return sorted(tuple(x) for x in groups.values())


def test_preprocess_order_and_reach(B, gen, orc):
    for g in undirected_graphs(gen):
        with B.BcmGraph.from_graph(g) as h:
            order, lo, hi = h.preprocess()
            comp, al, om, nc = h.scc_bounds()
        assert np.array_equal(order, orc.order(g)), g.name
        f, r = orc.farness_all(g)
        assert np.array_equal(lo, r) and np.array_equal(hi, r), g.name
        # undirected: the components are the SCCs of the symmetric digraph
        assert _partition(comp) == _partition(orc.scc(g)[0]), g.name
        assert nc == orc.scc(g)[1]
        # labels are numbered in order of each component's smallest member
        firsts = {}
        for v, c in enumerate(comp.tolist()):
            firsts.setdefault(c, v)
        assert sorted(firsts, key=firsts.get) == list(range(nc)), g.name


@pytest.mark.parametrize("lanes", LANES)
def test_farness_all_small(B, gen, orc, lanes):
    for g in undirected_graphs(gen):
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            gf, gr, st = h.farness_all(grid_lanes=lanes)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), (g.name, lanes)
            gf, gr, st = h.farness_all(lanes=lanes, flags=B.BCM_CTA_ONLY)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), (g.name, lanes, "cta")
            gf, gr, st = h.farness_all(grid_lanes=lanes, flags=B.BCM_ALL_PULL)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), (g.name, lanes, "pull")
            gf, gr, st = h.farness_all(grid_lanes=lanes, flags=B.BCM_NO_PULL)
            assert np.array_equal(gf, f) and np.array_equal(gr, r), (g.name, lanes, "push")


@pytest.mark.parametrize("lanes,threads", [(64, 256), (64, 512), (128, 512), (256, 256), (256, 1024)])
def test_topk_small(B, gen, orc, lanes, threads):
    for g in undirected_graphs(gen):
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            for k in sorted({1, 2, 3, 10, 100, min(g.n, 1024), min(g.n + 4, 1024)} - {0}):
                ids, gf, gr, st = h.topk(k, lanes=lanes, threads=threads)
                exp = orc.topk(f, r, k)
                assert np.array_equal(ids, exp), (g.name, k, lanes)
                assert np.array_equal(gf, f[exp]) and np.array_equal(gr, r[exp]), (g.name, k)
                assert st["completed"] + st["cut"] == g.n, (g.name, k, st)


def test_topk_kernel_choices_and_footnote(B, gen, orc):
    """Every wave on one kernel or the other, any grid width, the heavy/light
    switch at several points, and the bound without the undirected footnote."""
    for g in undirected_graphs(gen)[::2]:
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            for k in (1, 5, 40):
                exp = orc.topk(f, r, k)
                for flags in (B.BCM_CTA_ONLY, B.BCM_GRID_ONLY, B.BCM_NO_FOOTNOTE,
                              B.BCM_CTA_ONLY | B.BCM_NO_FOOTNOTE, B.BCM_GRID_ONLY | B.BCM_NO_FOOTNOTE):
                    ids, gf, gr, st = h.topk(k, flags=flags)
                    assert np.array_equal(ids, exp), (g.name, k, flags)
                for gl in (64, 128, 256):
                    for hw in (1, 50, 1 << 30):
                        ids, gf, gr, st = h.topk(k, grid_lanes=gl, heavy_words=hw)
                        assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]), (g.name, k, gl, hw)
                    # every grid level by pull, then every one by push
                    for flags, pd in ((B.BCM_GRID_ONLY | B.BCM_ALL_PULL, 0), (B.BCM_GRID_ONLY | B.BCM_NO_PULL, 0),
                                      (B.BCM_GRID_ONLY, 1 << 30)):
                        ids, gf, gr, st = h.topk(k, grid_lanes=gl, flags=flags, pull_div=pd)
                        assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]), (g.name, k, gl, pd)


def test_exhaustive_m_vis_is_the_push_count_either_way(B, gen):
    """m_vis of an exhaustive run is, summed over sources v, the out-degree
    of every vertex v reaches (v included): the arcs a push scans.  Pushed
    levels count it entry by entry, pulled ones from the lanes' counters;
    every direction choice, grid width and footnote setting must give this
    closed form (reachability from scipy's BFS)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    graphs = undirected_graphs(gen)[::2] + [gen.gnp(300, 0.01, seed=7, directed=True), gen.rmat(10, 8, seed=9),
                                            gen.with_self_loops_and_repeats(gen.ba(300, 3, seed=2), seed=3)]
    for g in graphs:
        deg = g.degrees()
        a = csr_matrix((np.ones(g.m), g.col.astype(np.int64), g.row_ptr.astype(np.int64)), shape=(g.n, g.n))
        exp = sum(int(deg[breadth_first_order(a, v, directed=True, return_predecessors=False)].sum())
                  for v in range(g.n))
        with B.BcmGraph.from_graph(g) as h:
            for gl in (64, 128, 256):
                for pd, flags in ((0, B.BCM_ALL_PULL), (0, B.BCM_ALL_PULL | B.BCM_NO_FOOTNOTE), (0, B.BCM_NO_PULL), (0, 0),
                                  (1 << 30, 0)):
                    _, _, st = h.farness_all(grid_lanes=gl, pull_div=pd, flags=flags)
                    assert st["m_vis"] == exp, (g.name, gl, pd, flags, st["m_vis"], exp)


def test_deferred_waves_rerun_exactly(B, gen, orc):
    """Per-CTA waves that hand their sources to the second grid-wide pass
    (forced with tiny defer_words) give the exact top-k: a deferred source is
    run again from the start under the threshold of the moment."""
    graphs = undirected_graphs(gen)[1::2] + [gen.gnp(300, 0.01, seed=7, directed=True), gen.rmat(10, 8, seed=9)]
    for g in graphs:
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            for k in (1, 10, 50):
                exp = orc.topk(f, r, k)
                for hw, dw, lanes in ((1 << 30, 1, 64), (1 << 30, 3, 256), (1, 2, 64), (50, 1, 128)):
                    ids, gf, gr, st = h.topk(k, heavy_words=hw, defer_words=dw, lanes=lanes)
                    assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]) and np.array_equal(gr, r[exp]), \
                        (g.name, k, hw, dw, lanes)
                    if hw == 1 << 30 and dw == 1 and g.m > 0 and g.n > 1:
                        assert st["deferred"] > 0, g.name
                ids, gf, gr, st = h.topk(k, heavy_words=1 << 30, defer_words=1, flags=B.BCM_NO_DEFER)
                assert np.array_equal(ids, exp) and st["deferred"] == 0


def test_prefilter_is_exact(B, gen, orc):
    """The level-0/1 prefilter (simple graphs, after grid-wide waves) stops
    sources from degrees alone; the top-k is the oracle's with or without
    it, and it cuts the sources the waves would have.  A graph with
    self-loops and repeated arcs is not simple: the prefilter stays off."""
    graphs = undirected_graphs(gen)[::3] + [gen.chung_lu(1 << 14, 10.0, 2.3, seed=9), gen.rmat(12, 8, seed=4),
                                            gen.gnp(400, 0.01, seed=8, directed=True),
                                            gen.with_self_loops_and_repeats(gen.ba(300, 3, seed=2), seed=3)]
    for g in graphs:
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            for k in (1, 10, 50):
                exp = orc.topk(f, r, k)
                for hw in (1, 64):                # grid-wide waves run, then the prefilter
                    a = h.topk(k, heavy_words=hw)
                    b = h.topk(k, heavy_words=hw, flags=B.BCM_NO_PREFILTER)
                    for ids, gf, gr, st in (a, b):
                        assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]) and \
                            np.array_equal(gr, r[exp]), (g.name, k, hw)
                    # every source ends once: completed or stopped (deferred ones are rerun)
                    for st in (a[3], b[3]):
                        assert st["completed"] + st["cut"] == g.n, (g.name, k, hw, st["completed"], st["cut"])


def test_plain_equals_oracle_bcm(B, gen, orc):
    """One source per launch follows the oracle's Algorithm 1 step for step:
    same top-k and the same arcs scanned, completions and cuts."""
    for g in undirected_graphs(gen)[:14] + [gen.ba(400, 3, seed=5)]:
        with B.BcmGraph.from_graph(g) as h:
            for k in (1, 3, 10):
                ids, gf, gr, st = h.topk(k, flags=B.BCM_PLAIN)
                oi, of, orr, ost = orc.bcm(g, k, early_test=True)
                assert np.array_equal(ids, oi) and np.array_equal(gf, of) and np.array_equal(gr, orr), (g.name, k)
                assert st["m_vis"] == ost["m_vis"], (g.name, k, st["m_vis"], ost["m_vis"])
                assert st["completed"] == ost["completed"] and st["cut"] == ost["cut"], (g.name, k)


@pytest.mark.parametrize("k", [1, 10, 100])
def test_workload_ba2000(B, gen, orc, k):
    g = gen.workload("ba2000")
    f, r = orc.farness_all(g)
    exp = orc.topk(f, r, k)
    with B.BcmGraph.from_graph(g) as h:
        for lanes in LANES:
            ids, gf, gr, st = h.topk(k, lanes=lanes)
            assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]) and np.array_equal(gr, r[exp])
        if k <= 10:
            ids, gf, gr, st = h.topk(k, flags=B.BCM_PLAIN)
            assert np.array_equal(ids, exp)
            assert st["m_vis"] == orc.bcm(g, k)[3]["m_vis"]
        gf, gr, _ = h.farness_all()
        assert np.array_equal(gf, f) and np.array_equal(gr, r)


@pytest.mark.parametrize("lanes", LANES)
def test_chunglu_16k(B, gen, orc, lanes):
    g = gen.chung_lu(1 << 14, 10.0, 2.3, seed=2)
    f, r = orc.farness_all(g)
    with B.BcmGraph.from_graph(g) as h:
        for k in (1, 10, 100):
            ids, gf, gr, st = h.topk(k, lanes=lanes)
            exp = orc.topk(f, r, k)
            assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]) and np.array_equal(gr, r[exp])
        gf, gr, _ = h.farness_all(lanes=lanes)
        assert np.array_equal(gf, f) and np.array_equal(gr, r)


def test_device_outputs(B, gen, orc):
    import torch
    g = gen.grid_lcc(40, 40, 0.05, seed=9)
    f, r = orc.farness_all(g)
    exp = orc.topk(f, r, 7)
    rp = torch.from_numpy(g.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(g.col.view(np.int32)).cuda()
    h = B.bcm_graph_create(rp, col, g.n, g.m, False, ptr_on_device=True)
    try:
        ids = torch.zeros(7, dtype=torch.int32, device="cuda")
        far = torch.zeros(7, dtype=torch.int64, device="cuda")
        reach = torch.zeros(7, dtype=torch.int32, device="cuda")
        B.bcm_topk(h, 7, B.make_options(flags=B.BCM_OUT_DEVICE), ids, far, reach)
        assert ids.cpu().numpy().view(np.uint32).tolist() == exp.tolist()
        assert far.cpu().numpy().view(np.uint64).tolist() == f[exp].tolist()
        fa = torch.zeros(g.n, dtype=torch.int64, device="cuda")
        ra = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        B.bcm_farness_all(h, B.make_options(flags=B.BCM_OUT_DEVICE), fa, ra)
        assert np.array_equal(fa.cpu().numpy().view(np.uint64), f)
        assert np.array_equal(ra.cpu().numpy().view(np.uint32), r)
    finally:
        B.bcm_graph_destroy(h)


def test_errors(B, gen):
    g = gen.path(5)
    with B.BcmGraph.from_graph(g) as h:
        for bad in (dict(k=0), dict(k=1025)):
            with pytest.raises(B.BcmError) as ei:
                h.topk(**bad)
            assert ei.value.status == B.BCM_ERR_INVALID
        with pytest.raises(B.BcmError) as ei:
            h.topk(1, lanes=32)
        assert ei.value.status == B.BCM_ERR_UNSUPPORTED
        with pytest.raises(B.BcmError) as ei:
            h.topk(1, lanes=256, threads=128)
        assert ei.value.status == B.BCM_ERR_UNSUPPORTED
        with pytest.raises(B.BcmError) as ei:
            h.topk(1, grid_lanes=96)
        assert ei.value.status == B.BCM_ERR_UNSUPPORTED
        with pytest.raises(B.BcmError) as ei:
            h.topk(1, flags=B.BCM_CTA_ONLY | B.BCM_GRID_ONLY)
        assert ei.value.status == B.BCM_ERR_INVALID
    bad_rp = np.array([0, 2, 1, 3], np.uint64)
    with pytest.raises(B.BcmError) as ei:
        B.BcmGraph(bad_rp, np.array([1, 2, 0], np.uint32), 3, False)
    assert ei.value.status == B.BCM_ERR_INVALID
    with pytest.raises(B.BcmError) as ei:
        B.BcmGraph(np.array([0, 1, 1], np.uint64), np.array([5], np.uint32), 2, False)
    assert ei.value.status == B.BCM_ERR_INVALID
    # an undirected graph whose arc 0->1 has no partner
    with pytest.raises(B.BcmError) as ei:
        B.BcmGraph(np.array([0, 1, 1], np.uint64), np.array([1], np.uint32), 2, False,
                   flags=B.BCM_CHECK_SYMMETRIC)
    assert ei.value.status == B.BCM_ERR_NOT_SYMMETRIC
    with B.BcmGraph.from_graph(gen.grid(3, 3), flags=B.BCM_CHECK_SYMMETRIC) as h:
        assert h.topk(1)[0].tolist() == [4]


def test_bounded_waits_time_out_cleanly(B, gen, orc):
    """Failure detection without a fault: a wait limit far below any real
    grid-barrier wait makes the waiting blocks give up.  The kernel records
    the error and every block leaves; the call returns BCM_ERR_TIMEOUT, and
    the next calls on the same handle and context are exact."""
    g = gen.chung_lu(1 << 15, 10.0, 2.3, seed=3)
    f, r = orc.farness_all(g)
    exp = orc.topk(f, r, 10)
    with B.BcmGraph.from_graph(g) as h:
        for _ in range(2):
            with pytest.raises(B.BcmError) as ei:
                h.topk(10, wait_limit_ns=1, flags=B.BCM_GRID_ONLY)
            assert ei.value.status == B.BCM_ERR_TIMEOUT
            assert "limit" in str(ei.value)
            ids, gf, gr, st = h.topk(10)
            assert np.array_equal(ids, exp) and np.array_equal(gf, f[exp]) and np.array_equal(gr, r[exp])
        with pytest.raises(B.BcmError) as ei:
            h.farness_all(wait_limit_ns=1)
        assert ei.value.status == B.BCM_ERR_TIMEOUT
        gf, gr, _ = h.farness_all()
        assert np.array_equal(gf, f) and np.array_equal(gr, r)


def test_repeated_runs_reuse_clean_workspace(B, gen, orc):
    g = gen.ba(500, 3, seed=21)
    f, r = orc.farness_all(g)
    with B.BcmGraph.from_graph(g) as h:
        for it in range(4):
            for k in (1, 17):
                ids, gf, gr, st = h.topk(k, lanes=LANES[it % 3])
                assert np.array_equal(ids, orc.topk(f, r, k))
            gf, gr, _ = h.farness_all(lanes=LANES[(it + 1) % 3])
            assert np.array_equal(gf, f)
