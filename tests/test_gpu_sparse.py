"""The one-source-per-CTA kernel (k_sparse: a visited bitmap and two vertex
queues per CTA) against the oracle, through the C-ABI.

* BCM_SPARSE top-k on every small graph family the parity tests use,
  undirected and directed, k = 1, 10, 100: ids, farness and reach equal the
  oracle's exhaustive top-k element by element.
* bcm_farness_all with BCM_SPARSE: every vertex's farness and reach.
* Lattices (undirected, largest degree <= 8, n >= 4096) take the kernel by
  default -- no grid-wide wave runs -- and give the oracle's answer, as do
  bit-lane waves forced on them (BCM_NO_SPARSE).
* A frontier longer than the queue (2^18 entries) hands its source to the
  grid-wide pass: forced on a power-law graph of 2^19 vertices, sources are
  deferred and the answer is still Algorithm 1's.
"""
import numpy as np
import pytest

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


def _small(gen):
    gs = [gen.path(9), gen.star(12), gen.cycle(11), gen.complete(7), gen.grid(5, 6), gen.empty(4), gen.path(1),
          gen.path(2), gen.disjoint_union(gen.cycle(5), gen.cycle(5), gen.empty(1), gen.cycle(5)),
          gen.relabel(gen.grid(4, 4), seed=5), gen.ba(200, 2, seed=11), gen.grid_lcc(12, 12, 0.1, seed=2),
          gen.with_self_loops_and_repeats(gen.grid(4, 5), seed=1), gen.star(300), gen.grid(17, 19),
          gen.complete(260), gen.ba(3000, 8, seed=12), gen.chung_lu(3000, 6.0, 2.3, seed=4)]
    for s in range(4):
        gs.append(gen.gnp(60 + 37 * s, 0.02 + 0.01 * s, seed=100 + s, directed=False))
        gs.append(gen.gnp(80 + 29 * s, 0.02 + 0.01 * s, seed=200 + s, directed=True))
    gs.append(gen.rmat(10, 8, seed=6))
    return gs


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_sparse_topk_small_graphs(B, gen, orc, threads):
    for g in _small(gen):
        with B.BcmGraph.from_graph(g) as h:
            for k in (1, 10, 100):
                exp = orc.topk_exhaustive(g, k)
                ids, far, reach, st = h.topk(k, flags=B.BCM_SPARSE, threads=threads)
                assert np.array_equal(ids, exp[0]) and np.array_equal(far, exp[1]) and \
                    np.array_equal(reach, exp[2]), (g.name, k, threads)
                assert st["grid_waves"] == 0, g.name


def test_sparse_farness_all(B, gen, orc):
    for g in _small(gen) + [gen.grid_lcc(64, 64, 0.05, seed=3)]:
        f, r = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            gf, gr, st = h.farness_all(flags=B.BCM_SPARSE)
        assert np.array_equal(gf, f) and np.array_equal(gr, r), g.name


def test_lattices_default_to_sparse(B, gen, orc):
    for g in [gen.grid_lcc(128, 128, 0.05, seed=4), gen.grid(70, 90), gen.grid_lcc(256, 200, 0.1, seed=5)]:
        with B.BcmGraph.from_graph(g) as h:
            for k in (1, 10, 100):
                ei, ef, er, _ = orc.bcm(g, k)
                ids, far, reach, st = h.topk(k)
                assert np.array_equal(ids, ei) and np.array_equal(far, ef) and np.array_equal(reach, er), (g.name, k)
                assert st["grid_waves"] == 0 and st["waves"] == g.n, (g.name, st)
                ids, far, reach, st = h.topk(k, flags=B.BCM_NO_SPARSE)
                assert np.array_equal(ids, ei) and np.array_equal(far, ef) and np.array_equal(reach, er), (g.name, k)


def test_queue_overflow_defers(B, gen, orc):
    g = gen.chung_lu(1 << 19, 10.0, 2.3, seed=6)
    ei, ef, er, _ = orc.bcm(g, 10)
    with B.BcmGraph.from_graph(g) as h:
        ids, far, reach, st = h.topk(10, flags=B.BCM_SPARSE)
    assert np.array_equal(ids, ei) and np.array_equal(far, ef) and np.array_equal(reach, er)
    assert st["deferred"] > 0, st


def test_sparse_flag_conflict(B, gen):
    with B.BcmGraph.from_graph(gen.grid(70, 70)) as h:
        with pytest.raises(B.BcmError):
            h.topk(10, flags=B.BCM_SPARSE | B.BCM_NO_SPARSE)
