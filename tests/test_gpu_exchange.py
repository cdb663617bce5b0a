"""The threshold exchange between shards on the GPU (Section 2: the threads of
the parallel version share x_k).

* Two shards of one graph run at once from two threads of this process
  (one GPU context; each shard its own handle and stream, as the serving
  loop runs graphs), with paper_1507_01490_gb300.exchange.ThresholdExchange
  over a ThreadGather between bcm_topk_start and the run's end: the keys
  travel on the host, no kernel waits for another, and the merged lists
  are the oracle's top-k.
* A run offered keys many times while it is pending (from another thread,
  as the exchange does) stays exact: every block of a grid-wide launch cuts
  with the same snapshot of the threshold.
"""
import threading

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


def _graphs(gen):
    return [gen.chung_lu(1 << 15, 10.0, 2.3, seed=2), gen.rmat(13, 8, seed=3), gen.ba(20000, 4, seed=8)]


@pytest.mark.parametrize("k", [1, 10])
def test_two_shards_exchange_on_the_gpu(B, gen, orc, k):
    import torch
    from paper_1507_01490_gb300.exchange import ThreadGather, ThresholdExchange
    world = 2
    for g in _graphs(gen):
        tg = ThreadGather(world)
        lists, rounds, errs = [None] * world, [0] * world, []
        handles = [B.BcmGraph.from_graph(g) for _ in range(world)]
        try:
            for h in handles:
                h.preprocess()

            def rank_main(rank):
                try:
                    torch.cuda.set_device(0)
                    h = handles[rank]
                    kk = max(min(k, B.shard_size(g.n, rank, world)), 1)
                    ids = np.zeros(kk, np.uint32)
                    far = np.zeros(kk, np.uint64)
                    reach = np.zeros(kk, np.uint32)
                    B.bcm_topk_start(h.h, k, B.make_options(shard_index=rank, shard_count=world), ids, far, reach)
                    ex = ThresholdExchange(period_s=0, gather=tg.for_rank(rank))
                    ex.run(lambda: B.bcm_topk_threshold(h.h), lambda key: B.bcm_topk_offer(h.h, key),
                           lambda: B.bcm_topk_finish(h.h, wait=False))
                    lists[rank] = (ids, far, reach)
                    rounds[rank] = ex.rounds
                except BaseException as e:   # reported by the main thread
                    errs.append(e)
                    tg.bar.abort()

            ts = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
            for t in ts:
                t.start()
            for t in ts:
                t.join()
        finally:
            for h in handles:
                h.close()
        assert not errs, errs
        exp_ids, exp_f, exp_r = orc.topk_exhaustive(g, k)
        mi, mf, mr = B.bcm_topk_merge(np.concatenate([x[0] for x in lists]), np.concatenate([x[1] for x in lists]),
                                      np.concatenate([x[2] for x in lists]), k)
        assert np.array_equal(mi, exp_ids) and np.array_equal(mf, exp_f) and np.array_equal(mr, exp_r), g.name
        assert min(rounds) >= 1


def _key(f, r, v):
    return (1, (int(r) - 1) ** 2, int(f), int(v)) if r > 1 and f > 0 else (1, 0, 1, int(v))


def test_offers_during_a_run_keep_it_exact(B, gen, orc):
    """A thread keeps offering stronger keys while the run is pending -- the
    keys of the graph's entries ranked k+60 down to k, each a valid threshold,
    arriving at any moment -- and the shard lists still merge to the oracle's
    top-k."""
    g = gen.chung_lu(1 << 16, 10.0, 2.3, seed=12)
    k = 10
    f, r = orc.farness_all(g)
    ranked = orc.topk(f, r, k + 60)
    exp = ranked[:k]
    keys = [_key(f[v], r[v], v) for v in ranked[k - 1:][::-1]]   # weakest first, the k-th last
    with B.BcmGraph.from_graph(g) as h:
        for rep in range(3):
            lists = []
            for i in range(2):
                kk = min(k, B.shard_size(g.n, i, 2))
                ids = np.zeros(kk, np.uint32)
                far = np.zeros(kk, np.uint64)
                reach = np.zeros(kk, np.uint32)
                B.bcm_topk_start(h.h, k, B.make_options(shard_index=i, shard_count=2, grid_lanes=64), ids, far,
                                 reach)
                stop = threading.Event()

                def offer():
                    for key in keys:
                        if stop.is_set():
                            return
                        try:
                            B.bcm_topk_offer(h.h, key)
                        except B.BcmError:
                            return            # the run finished
                t = threading.Thread(target=offer)
                t.start()
                try:
                    B.bcm_topk_finish(h.h, wait=True)
                finally:
                    stop.set()
                    t.join()
                lists.append((ids, far, reach))
            mi, mf, mr = B.bcm_topk_merge(np.concatenate([x[0] for x in lists]),
                                          np.concatenate([x[1] for x in lists]),
                                          np.concatenate([x[2] for x in lists]), k)
            assert np.array_equal(mi, exp) and np.array_equal(mf, f[exp]) and np.array_equal(mr, r[exp]), rep
