"""bcm_topk over one shard of the sources: every shard of a graph run on this
GPU in turn, their lists merged by bcm_topk_merge, equals the graph's top-k
from the oracle (bit-exact)."""
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


def test_shards_merge_to_the_topk(B, gen, orc):
    graphs = [gen.ba(2000, 3, seed=1), gen.chung_lu(1 << 15, 10.0, 2.3, seed=2), gen.rmat(13, 8, seed=3),
              gen.grid_lcc(50, 50, 0.05, seed=4), gen.disjoint_union(gen.cycle(7), gen.empty(3), gen.star(9))]
    for g in graphs:
        f, r = orc.farness_all(g)
        order = orc.order(g)
        with B.BcmGraph.from_graph(g) as h:
            for count in (2, 3, 8):
                for k in (1, 10, 100):
                    lists = []
                    for i in range(count):
                        ids, far, reach, st = h.topk(k, shard_index=i, shard_count=count)
                        mine = order[B.shard_positions(g.n, i, count)]
                        assert len(ids) == min(k, len(mine))
                        assert np.isin(ids, mine).all()
                        # the shard's own top-k, exactly (the oracle breaks ties by array
                        # position, so it gets the shard's vertices in id order)
                        sm = np.sort(mine)
                        exp_i = sm[orc.topk(f[sm], r[sm], k)]
                        assert np.array_equal(ids, exp_i), (g.name, count, i, k)
                        lists.append((ids, far, reach))
                    mi, mf, mr = B.bcm_topk_merge(np.concatenate([x[0] for x in lists]),
                                                  np.concatenate([x[1] for x in lists]),
                                                  np.concatenate([x[2] for x in lists]), k)
                    exp = orc.topk(f, r, k)
                    assert np.array_equal(mi, exp) and np.array_equal(mf, f[exp]) and np.array_equal(mr, r[exp])


def test_shard_arguments(B, gen):
    with B.BcmGraph.from_graph(gen.path(5)) as h:
        with pytest.raises(B.BcmError) as ei:
            h.topk(1, shard_index=2, shard_count=2)
        assert ei.value.status == B.BCM_ERR_INVALID
        ids, _, _, _ = h.topk(3, shard_index=1, shard_count=2)   # 5 positions: shard 1 is empty
        assert len(ids) == 0


def _key(f, r, v):
    return (1, 0, 1, int(v)) if r <= 1 or f == 0 else (1, (int(r) - 1) ** 2, int(f), int(v))


def test_offered_key_keeps_the_topk(B, gen, orc):
    """Each shard's run is offered the graph's exact k-th key (what the
    threshold exchange converges to) while it is pending: its list (padding
    aside) still holds every top-k member of its shard with the oracle's
    farness and reach, the merge is the graph's top-k, and the read-back
    threshold of a run is its k-th entry's key."""
    graphs = [gen.ba(2000, 3, seed=1), gen.chung_lu(1 << 15, 10.0, 2.3, seed=2), gen.rmat(13, 8, seed=3),
              gen.grid_lcc(50, 50, 0.05, seed=4)]
    for g in graphs:
        f, r = orc.farness_all(g)
        order = orc.order(g)
        with B.BcmGraph.from_graph(g) as h:
            with pytest.raises(B.BcmError) as ei:
                B.bcm_topk_offer(h.h, (1, 1, 1, 0))      # no run pending
            assert ei.value.status == B.BCM_ERR_INVALID
            for count in (2, 3):
                for k in (1, 10, 100):
                    exp = orc.topk(f, r, k)
                    kth = _key(f[exp[-1]], r[exp[-1]], exp[-1])
                    lists = []
                    for i in range(count):
                        kk = max(min(k, B.shard_size(g.n, i, count)), 1)
                        ids = np.zeros(kk, np.uint32)
                        far = np.zeros(kk, np.uint64)
                        reach = np.zeros(kk, np.uint32)
                        opts = B.make_options(shard_index=i, shard_count=count)
                        B.bcm_topk_start(h.h, k, opts, ids, far, reach)
                        B.bcm_topk_offer(h.h, kth)
                        B.bcm_topk_offer(h.h, (1, 1, 10**12, 5))   # weaker than kth: ignored
                        assert B.bcm_topk_finish(h.h, wait=True)
                        real = ids != B.PAD_ID
                        assert (far[~real] == 0).all() and (reach[~real] == 0).all()
                        ri, rf, rr = ids[real], far[real], reach[real]
                        assert np.array_equal(rf, f[ri]) and np.array_equal(rr, r[ri]), (g.name, count, i, k)
                        mine = set(order[B.shard_positions(g.n, i, count)].tolist())
                        assert set(exp.tolist()) & mine <= set(ri.tolist()), (g.name, count, i, k)
                        lists.append((ids, far, reach))
                    mi, mf, mr = B.bcm_topk_merge(np.concatenate([x[0] for x in lists]),
                                                  np.concatenate([x[1] for x in lists]),
                                                  np.concatenate([x[2] for x in lists]), k)
                    assert np.array_equal(mi, exp) and np.array_equal(mf, f[exp]) and np.array_equal(mr, r[exp])
            ids, far, reach, _ = h.topk(10)
            assert B.bcm_topk_threshold(h.h) == _key(far[-1], reach[-1], ids[-1])
