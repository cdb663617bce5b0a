"""bcm_farness_all_noalloc, the entry point that allocates nothing.

It is for callers that cannot allocate device memory when they need the
result (a host framework owning all device memory, a request path that must
not pay an allocation's device synchronisation, a fixed memory budget).  Its
working memory is a fixed array inside the library, so these tests check
that two calls in a row, which reuse that array, each give exactly what
bcm_farness_all gives and what the oracle's plain BFS from every vertex
gives.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_N = 1_250_000   # the entry point's documented vertex limit


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


def _on_device(g):
    import torch
    rp = torch.from_numpy(g.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy((g.col if g.m else np.zeros(1, np.uint32)).view(np.int32)).cuda()
    return rp, col


def _two_calls(B, g, expect_f, expect_r):
    import torch
    rp, col = _on_device(g)
    for call in range(2):
        far = torch.full((g.n,), -1, dtype=torch.int64, device="cuda")
        reach = torch.full((g.n,), -1, dtype=torch.int32, device="cuda")
        B.bcm_farness_all_noalloc(rp, col, g.n, g.m, None, far, reach)
        torch.cuda.synchronize()
        assert np.array_equal(far.cpu().numpy().view(np.uint64), expect_f), (g.name, call)
        assert np.array_equal(reach.cpu().numpy().view(np.uint32), expect_r), (g.name, call)


def test_two_calls_match_farness_all_and_oracle(B, gen, orc):
    graphs = [gen.ba(2000, 3, seed=1), gen.chung_lu(1 << 14, 10.0, 2.3, seed=2), gen.rmat(12, 8, seed=3),
              gen.grid_lcc(60, 60, 0.05, seed=4), gen.disjoint_union(gen.cycle(7), gen.empty(3), gen.star(9))]
    for g in graphs:
        of, orr = orc.farness_all(g)
        with B.BcmGraph.from_graph(g) as h:
            ef, er, _ = h.farness_all()
        assert np.array_equal(ef, of) and np.array_equal(er, orr), g.name
        _two_calls(B, g, of, orr)


def test_at_the_vertex_limit(B, gen, orc):
    """n at the limit, where one wave slot is all the array holds: 125,000
    paths of 10 vertices (every BFS stays in its path, so the oracle's
    complete answer takes a second)."""
    n = MAX_N
    i = np.arange(n, dtype=np.int64)
    keep = (i % 10) != 9
    g = gen.csr_from_arcs(n, i[keep], i[keep] + 1, directed=False, name="paths10x125000")
    of, orr = orc.farness_all(g)
    assert (orr == 10).all()
    _two_calls(B, g, of, orr)


def test_rejects_graphs_beyond_its_limit(B):
    import torch
    rp = torch.zeros(4, dtype=torch.int64, device="cuda")
    col = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(B.BcmError) as ei:
        B.bcm_farness_all_noalloc(rp, col, MAX_N + 1, 0, None, out, col)
    assert ei.value.status == B.BCM_ERR_UNSUPPORTED
    assert str(MAX_N) in str(ei.value)
