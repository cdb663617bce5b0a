"""Per-CTA vertex tables against the oracle (Algorithm 1 with BFSCut).

A per-CTA wave keeps its vertices' bit words in a table: dense (vertex x
is entry x) on graphs no larger than the table, hashed (linear probing,
2^16 entries by default) on larger ones, where a wave that makes more than
half as many entries is handed to the grid-wide pass like a wide wave.

* Hashed tables of several sizes -- down to 1,024 entries, which most waves
  overflow -- and the dense layout give the oracle's top-k element by
  element, on graphs where the per-CTA waves do most of the work
  (Barabasi-Albert), where the prefilter leaves them little (Chung-Lu), on
  a digraph (R-MAT) and on a high-diameter lattice (deep waves).
* A small table defers waves (the counters say so) and its workspace is
  smaller than the dense one.
* Options outside the supported range are refused.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DENSE = 1 << 30   # a table at least n: the dense layout


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
    return [gen.ba(100000, 4, seed=21), gen.chung_lu(1 << 17, 10.0, 2.3, seed=5), gen.rmat(16, 8, seed=7),
            gen.grid_lcc(320, 320, 0.1, seed=9)]


@pytest.fixture(scope="module")
def cases(gen, orc):
    out = []
    for g in _graphs(gen):
        exp = {k: orc.bcm(g, k, refined=g.directed)[:3] for k in (1, 10, 100)}
        out.append((g, exp))
    return out


@pytest.mark.parametrize("table", [0, 1024, 4096, DENSE])
def test_tables_give_the_oracle_topk(B, cases, table):
    for g, exp in cases:
        with B.BcmGraph.from_graph(g) as h:
            for k, (ei, ef, er) in exp.items():
                for lanes in (64, 256):
                    ids, far, reach, st = h.topk(k, lanes=lanes, cta_table=table)
                    assert np.array_equal(ids, ei) and np.array_equal(far, ef) and np.array_equal(reach, er), \
                        (g.name, k, table, lanes)


def test_small_table_defers_and_shrinks_the_workspace(B, gen, orc):
    g = gen.ba(100000, 4, seed=21)
    ei, ef, er, _ = orc.bcm(g, 10)
    with B.BcmGraph.from_graph(g) as h:
        ws = {t: B.bcm_workspace_bytes(h.h, B.make_options(cta_table=t)) for t in (1024, 0, DENSE)}
        assert ws[1024] < ws[0] < ws[DENSE]
        _, _, _, dense = h.topk(10, cta_table=DENSE)
        ids, far, reach, small = h.topk(10, cta_table=1024)
        assert np.array_equal(ids, ei) and np.array_equal(far, ef) and np.array_equal(reach, er)
        assert small["deferred"] > dense["deferred"]
        # with deferral off the table is dense whatever its size: same answer, same workspace
        ws_nd = B.bcm_workspace_bytes(h.h, B.make_options(cta_table=1024, flags=B.BCM_NO_DEFER))
        assert ws_nd == B.bcm_workspace_bytes(h.h, B.make_options(cta_table=DENSE, flags=B.BCM_NO_DEFER))
        ids, far, reach, _ = h.topk(10, cta_table=1024, flags=B.BCM_NO_DEFER)
        assert np.array_equal(ids, ei) and np.array_equal(far, ef) and np.array_equal(reach, er)


def test_table_option_range(B, gen):
    g = gen.ba(30000, 3, seed=2)
    with B.BcmGraph.from_graph(g) as h:
        for bad in (512, 3000, 1 << 14 | 1):
            with pytest.raises(B.BcmError):
                h.topk(10, cta_table=bad)
        h.topk(10, cta_table=40000)   # not a power of two, but at least n: dense
