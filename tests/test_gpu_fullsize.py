"""Full-size workloads, in the launch configuration bench.py uses (library
defaults).

Complete check: tests/golden/fullsize_<workload>_k<k>.json hold the exact
top-k of chunglu1m and rmat20 (k = 1, 10, 100) and of the damaged-grid recipe
at 512 x 512 and 1024 x 1024 (k = 10) as the oracle's sequential Algorithm 1 computed it
(tests/golden/make_fullsize.py, which calls only the oracle); the GPU's ids,
farness and reach must equal them element by element.

The oracle cannot run every BFS of a million-vertex graph inside a test, so
the remaining checks are on sampled outputs it computes one by one:

* the k returned vertices: farness and reach equal one oracle BFS each;
* no sampled vertex (the highest-degree ones, where the top-k lives, plus a
  uniform sample) ranks above the k-th entry under the exact order;
* every returned entry ranks at or above every sampled non-entry, and the
  entries are in rank order;
* directed: the SCC partition, alpha and omega equal the oracle's on the
  whole graph (Tarjan and the Section 2.3 programme are cheap on the CPU),
  and sampled r(v) lie in [alpha(v), omega(v)].
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name, k):
    p = os.path.join(GOLDEN, "fullsize_%s_k%d.json" % (name, k))
    if not os.path.exists(p):
        pytest.fail("missing golden %s (tests/golden/make_fullsize.py writes it)" % p)
    return json.load(open(p))


def _check_golden(gold, g, ids, far, reach):
    assert gold["csr_sha256_16"] == g.hash64(), "the workload generator no longer makes the golden's graph"
    assert gold["n"] == g.n and gold["m"] == g.m
    assert ids.tolist() == gold["ids"]
    assert far.tolist() == gold["farness"]
    assert reach.tolist() == gold["reach"]


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


def _key(f, r):
    return (0, 1) if r <= 1 else ((r - 1) ** 2, f)


def _before(a, b):
    """a = (f, r, id) ranks strictly before b"""
    (Na, Fa), (Nb, Fb) = _key(a[0], a[1]), _key(b[0], b[1])
    if Na * Fb != Nb * Fa:
        return Na * Fb > Nb * Fa
    return a[2] < b[2]


def _check_topk(orc, gen, g, ids, far, reach, n_top=512, n_rand=512, seed=5):
    of, orr = orc.farness_all(g, sources=ids)
    assert np.array_equal(of, far) and np.array_equal(orr, reach), "returned farness/reach"
    ent = [(int(f), int(r), int(v)) for f, r, v in zip(far, reach, ids)]
    for a, b in zip(ent, ent[1:]):
        assert _before(a, b), "entries out of rank order"
    deg = g.degrees()
    cand = np.argsort(-deg, kind="stable")[:n_top].astype(np.uint32)
    sample = np.setdiff1d(np.concatenate([cand, gen.uniform_u32(seed, n_rand, g.n)]), ids)
    sf, sr = orc.farness_all(g, sources=sample)
    kth = ent[-1]
    for f, r, v in zip(sf, sr, sample):
        assert not _before((int(f), int(r), int(v)), kth), ("vertex %d beats the k-th" % v)
    return sample, sr


@pytest.fixture(scope="module")
def chunglu(gen):
    return gen.workload("chunglu1m")


@pytest.mark.parametrize("k", [1, 10, 100])
def test_chunglu1m(B, gen, orc, chunglu, k):
    g = chunglu
    with B.BcmGraph.from_graph(g) as h:
        ids, far, reach, st = h.topk(k)
    assert len(ids) == k
    _check_golden(_golden("chunglu1m", k), g, ids, far, reach)
    _check_topk(orc, gen, g, ids, far, reach)
    assert st["m_vis"] < 0.01 * g.m * g.n


def test_chunglu1m_lane_widths_agree(B, chunglu):
    """Every lane width of either kernel gives the oracle's exact top-100."""
    g = chunglu
    gold = _golden("chunglu1m", 100)
    with B.BcmGraph.from_graph(g) as h:
        for lanes in (64, 128, 256):
            for grid_lanes in (64, 256):
                ids, far, reach, _ = h.topk(100, lanes=lanes, grid_lanes=grid_lanes)
                _check_golden(gold, g, ids, far, reach)


@pytest.fixture(scope="module")
def rmat(gen):
    return gen.workload("rmat20")


def test_rmat20_scc_and_bounds(B, gen, orc, rmat):
    g = rmat
    ocomp, oal, oom, onc = orc.alpha_omega_refined(g)
    with B.BcmGraph.from_graph(g) as h:
        comp, al, om, nc = h.scc_bounds()
    assert nc == onc
    # same partition: labels map one-to-one
    pairs = np.unique((comp.astype(np.uint64) << np.uint64(32)) | ocomp.astype(np.uint64))
    assert pairs.size == nc
    assert np.array_equal(al, oal) and np.array_equal(om, oom)
    sample = gen.uniform_u32(11, 2000, g.n)
    f, r = orc.farness_all(g, sources=sample)
    assert (al[sample] <= r).all() and (r <= om[sample]).all()


@pytest.mark.parametrize("k", [1, 10, 100])
def test_rmat20_topk(B, gen, orc, rmat, k):
    g = rmat
    with B.BcmGraph.from_graph(g) as h:
        ids, far, reach, st = h.topk(k)
    _check_golden(_golden("rmat20", k), g, ids, far, reach)
    _check_topk(orc, gen, g, ids, far, reach)


def test_grid512_topk10(B, gen, orc):
    """The damaged-grid recipe at 512 x 512, against the oracle's complete
    answer (golden): BCM scans about 57% of m*n on such grids (the bound only
    bites late on a lattice), so the work grows with n^2; the graph's largest
    degree is 4, so it runs on the one-source kernel by default, and is also
    checked on bit-lane waves.  The 2048 x 2048 case is the opt-in test below."""
    g = gen.workload("grid512")
    gold = _golden("grid512", 10)
    with B.BcmGraph.from_graph(g) as h:
        ids, far, reach, st = h.topk(10)
        assert st["sparse"] == g.n and st["grid_waves"] == 0
        lanes = h.topk(10, flags=B.BCM_NO_SPARSE)
    _check_golden(gold, g, ids, far, reach)
    _check_golden(gold, g, *lanes[:3])
    _check_topk(orc, gen, g, ids, far, reach, n_top=64, n_rand=192)


def test_grid1024_topk10(B, gen):
    """The damaged-grid recipe at 1024 x 1024 (1,048,568 vertices, BFSs of up to
    about 1,900 levels) against the oracle's complete answer (a golden: 3.4 hours
    of the oracle's Algorithm 1 on one core); about 24 s on the GPU."""
    g = gen.workload("grid1024")
    gold = _golden("grid1024", 10)
    with B.BcmGraph.from_graph(g) as h:
        ids, far, reach, st = h.topk(10)
    assert st["sparse"] == g.n and st["grid_waves"] == 0
    _check_golden(gold, g, ids, far, reach)


@pytest.mark.skipif(not __import__("os").environ.get("BCM_TEST_GRID2048"),
                    reason="minutes of GPU time; set BCM_TEST_GRID2048=1")
def test_grid2048_topk10(B, gen, orc):
    g = gen.workload("grid2048")
    assert g.n > 4_000_000 and g.meta["deleted_edges"] == 419226
    with B.BcmGraph.from_graph(g) as h:
        ids, far, reach, st = h.topk(10)
    assert st["sparse"] == g.n
    assert (reach == g.n).all()
    _check_topk(orc, gen, g, ids, far, reach, n_top=64, n_rand=192)
