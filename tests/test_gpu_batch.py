"""bcm_batch_*: the top-k runs of many small graphs recorded as one CUDA graph
and replayed; every replay gives, for every graph, what bcm_topk gives."""
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


def small_graphs(gen):
    gs = []
    for i in range(12):
        gs.append(gen.ba(300 + 400 * i, 2 + i % 4, seed=50 + i))
        gs.append(gen.rmat(8 + i % 5, 4 + i % 6, seed=70 + i))
    gs += [gen.grid_lcc(40, 40, 0.05, seed=3), gen.disjoint_union(gen.cycle(9), gen.star(30), gen.empty(4)),
           gen.gnp(500, 0.01, seed=4, directed=True), gen.path(7), gen.complete(12)]
    return gs


def test_batch_replays_match_topk(B, gen, orc):
    import torch
    gs = small_graphs(gen)
    hs = [B.BcmGraph.from_graph(g) for g in gs]
    try:
        ks = [[1, 10, 100][i % 3] for i in range(len(gs))]
        exp = []
        for g, h, k in zip(gs, hs, ks):
            f, r = orc.farness_all(g)
            ids = orc.topk(f, r, k)
            exp.append((ids, f[ids], r[ids]))
            got = h.topk(k)
            assert np.array_equal(got[0], ids), g.name
        outs = [(torch.zeros(k, dtype=torch.int32, device="cuda"), torch.zeros(k, dtype=torch.int64, device="cuda"),
                 torch.zeros(k, dtype=torch.int32, device="cuda")) for k in ks]
        s = torch.cuda.Stream()
        batch = B.BcmBatch([h.h for h in hs], ks, outs, s)
        for rep in range(3):
            for o in outs:
                for t in o:
                    t.fill_(-1)
            torch.cuda.synchronize()
            batch.run()
            for (ids, f, r), o, g, k in zip(exp, outs, gs, ks):
                kk = min(k, g.n)
                assert np.array_equal(o[0][:kk].cpu().numpy().view(np.uint32), ids), (rep, g.name)
                assert np.array_equal(o[1][:kk].cpu().numpy().view(np.uint64), f), (rep, g.name)
                assert np.array_equal(o[2][:kk].cpu().numpy().view(np.uint32), r), (rep, g.name)
        batch.close()
        # the handles still work on their own afterwards
        assert np.array_equal(hs[0].topk(ks[0])[0], exp[0][0])
    finally:
        for h in hs:
            h.close()


def test_batch_rejects_large_graphs(B, gen):
    import torch
    big = gen.chung_lu(1 << 15, 10.0, 2.3, seed=2)
    with B.BcmGraph.from_graph(big) as h:
        o = (torch.zeros(10, dtype=torch.int32, device="cuda"), torch.zeros(10, dtype=torch.int64, device="cuda"),
             torch.zeros(10, dtype=torch.int32, device="cuda"))
        with pytest.raises(B.BcmError) as ei:
            B.BcmBatch([h.h], [10], [o], torch.cuda.Stream())
        assert ei.value.status == B.BCM_ERR_UNSUPPORTED
