"""Source sharding across GPUs (one graph, N ranks), on the CPU: the shard
rule partitions the degree order, bcm_topk_merge is the exact ranking, and
the N>1 host path -- each rank's shard top-k, one all-gather, the merge --
gives the graph's top-k, run as two gloo ranks, also with the ranks sharing
their k-th keys while they run (paper_1507_01490_gb300.exchange).  The
per-rank top-k comes from the oracle here (no GPU); the GPU side is
test_gpu_shard.py."""
import os
import socket

import numpy as np
import pytest

from paper_1507_01490_gb300 import bcm as B


@pytest.fixture(scope="module")
def lib():
    from paper_1507_01490_gb300 import _build
    _build.build_cuda()
    return B.load()


@pytest.mark.parametrize("n", [0, 1, 63, 64, 65, 200, 1000, 4097])
@pytest.mark.parametrize("count", [1, 2, 3, 8])
def test_shards_partition_the_order(n, count):
    seen = np.concatenate([B.shard_positions(n, i, count) for i in range(count)]) if n else np.array([])
    assert sorted(seen.tolist()) == list(range(n))
    for i in range(count):
        pos = B.shard_positions(n, i, count)
        assert len(pos) == B.shard_size(n, i, count)
        assert (np.diff(pos) > 0).all()
        if count > 1:
            assert ((pos // B.SHARD_CHUNK) % count == i).all()


def _random_entries(seed, n):
    rng = np.random.default_rng(seed)
    r = rng.integers(1, 40, n).astype(np.uint32)
    f = np.where(r > 1, rng.integers(1, 300, n), 0).astype(np.uint64)
    # plant exact ties of the score (r-1)^2 / f with different ids
    f[: n // 4] = ((r[: n // 4].astype(np.uint64) - 1) ** 2) * 3
    r[n // 4: n // 3] = 1
    f[n // 4: n // 3] = 0
    return f, r


@pytest.mark.parametrize("seed", range(6))
def test_merge_is_the_exact_ranking(lib, orc, seed):
    n = 500 + 37 * seed
    f, r = _random_entries(seed, n)
    ids = np.arange(n, dtype=np.uint32)
    perm = np.random.default_rng(100 + seed).permutation(n)
    for k in (1, 10, 100, n, n + 5):
        exp = orc.topk(f, r, k)
        oi, of, orr = B.bcm_topk_merge(ids[perm], f[perm], r[perm], k)
        assert np.array_equal(oi, exp), k
        assert np.array_equal(of, f[exp]) and np.array_equal(orr, r[exp])
        # merging per-part lists gives the same (each part's top-k holds its share of the answer)
        parts = np.array_split(perm, 3)
        lists = [orc.topk(f[p], r[p], k) for p in parts]
        cat = np.concatenate([p[l] for p, l in zip(parts, lists)]).astype(np.uint32)
        oi2, _, _ = B.bcm_topk_merge(cat, f[cat], r[cat], k)
        assert np.array_equal(oi2, exp), k


def test_merge_arguments(lib):
    with pytest.raises(B.BcmError) as ei:
        B.bcm_topk_merge([1], [2], [3], 0)
    assert ei.value.status == B.BCM_ERR_INVALID
    oi, of, orr = B.bcm_topk_merge([], [], [], 5)
    assert len(oi) == 0
    # padding of a shard list that holds fewer than k entries is skipped
    oi, of, orr = B.bcm_topk_merge([5, B.PAD_ID, 2, B.PAD_ID], [10, 0, 4, 0], [3, 0, 3, 0], 3)
    assert oi.tolist() == [2, 5] and of.tolist() == [4, 10] and orr.tolist() == [3, 3]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, k, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1507_01490_gb300 import graphgen
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for gi, g in enumerate([graphgen.ba(2000, 3, seed=1), graphgen.gnp(700, 0.006, seed=3, directed=True),
                                graphgen.disjoint_union(graphgen.cycle(40), graphgen.star(90), graphgen.path(70))]):
            order = oracle.order(g)
            # this shard's vertices, in id order (the oracle breaks ties by array position)
            mine = np.sort(order[B.shard_positions(g.n, rank, world)])
            f, r = oracle.farness_all(g, sources=mine)
            top = oracle.topk(f, r, k)                    # this shard's own top-k (positions in `mine`)
            local = (mine[top].astype(np.uint32), f[top], r[top])
            lists = [None] * world
            dist.all_gather_object(lists, local)
            ids = np.concatenate([x[0] for x in lists]).astype(np.uint32)
            far = np.concatenate([x[1] for x in lists]).astype(np.uint64)
            rch = np.concatenate([x[2] for x in lists]).astype(np.uint32)
            mi, mf, mr = B.bcm_topk_merge(ids, far, rch, k)
            fa, ra = oracle.farness_all(g)
            exp = oracle.topk(fa, ra, k)
            ok = np.array_equal(mi, exp) and np.array_equal(mf, fa[exp]) and np.array_equal(mr, ra[exp])
            with open(os.path.join(out_dir, "rank%d_graph%d" % (rank, gi)), "w") as fh:
                fh.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k", [1, 10, 64])
def test_two_gloo_ranks_merge_to_the_global_topk(lib, orc, tmp_path, k):
    import torch.multiprocessing as mp
    orc.build()
    mp.spawn(_rank_main, args=(2, _free_port(), k, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        for gi in range(3):
            assert (tmp_path / ("rank%d_graph%d" % (rank, gi))).read_text() == "ok", (rank, gi)


def test_key_order():
    from paper_1507_01490_gb300.exchange import NO_KEY, best_key, key_before
    a = (1, 16, 40, 7)       # (r-1)^2 / f = 0.4
    b = (1, 9, 30, 3)        # 0.3
    tie = (1, 32, 80, 5)     # 0.4, smaller id than a
    assert key_before(a, b) and not key_before(b, a)
    assert key_before(tie, a) and not key_before(a, tie)
    assert key_before(b, NO_KEY) and not key_before(NO_KEY, b) and not key_before(NO_KEY, NO_KEY)
    assert best_key([b, NO_KEY, a, tie]) == tie and best_key([]) == NO_KEY


def _exchange_rank_main(rank, world, port, k, chunk, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_1507_01490_gb300 import graphgen
    from paper_1507_01490_gb300.exchange import ThresholdExchange
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        graphs = [graphgen.ba(2000, 3, seed=1), graphgen.chung_lu(3000, 8.0, 2.3, seed=5),
                  graphgen.gnp(700, 0.006, seed=3, directed=True), graphgen.rmat(11, 8, seed=6)]
        offers = 0
        for gi, g in enumerate(graphs):
            order = oracle.order(g)
            src = order[B.shard_positions(g.n, rank, world)]
            if g.directed:
                _, al, om, _ = oracle.alpha_omega(g)
                bounds = (al, om)
            else:
                _, rr = oracle.farness_all(g)
                bounds = (rr, rr)
            alone = oracle.ShardRun(g, k, src, bounds)
            alone.step(len(src) + 1)
            run = oracle.ShardRun(g, k, src, bounds)
            ex = ThresholdExchange(period_s=0)
            ex.run(run.key, run.offer, lambda: run.step(chunk))
            offers += ex.offers
            ids, f, r, st = run.result()
            lists = [None] * world
            dist.all_gather_object(lists, (ids, f, r))
            mi, mf, mr = B.bcm_topk_merge(np.concatenate([x[0] for x in lists]),
                                          np.concatenate([x[1] for x in lists]),
                                          np.concatenate([x[2] for x in lists]), k)
            fa, ra = oracle.farness_all(g)
            exp = oracle.topk(fa, ra, k)
            ok = np.array_equal(mi, exp) and np.array_equal(mf, fa[exp]) and np.array_equal(mr, ra[exp])
            fewer = st["m_vis"] <= alone.result()[3]["m_vis"]
            with open(os.path.join(out_dir, "x_rank%d_graph%d" % (rank, gi)), "w") as fh:
                fh.write("ok" if ok and fewer else "mismatch %s %s" % (ok, fewer))
        with open(os.path.join(out_dir, "x_rank%d_offers" % rank), "w") as fh:
            fh.write(str(offers))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k", [1, 10])
def test_two_gloo_ranks_exchange_thresholds(lib, orc, tmp_path, k):
    """Two ranks, each running Algorithm 1 over its shard (the oracle, a few
    sources at a time), share their k-th keys every round: the merged top-k
    is the graph's, no rank scans more arcs than it would alone, and keys
    were actually offered."""
    import torch.multiprocessing as mp
    orc.build()
    mp.spawn(_exchange_rank_main, args=(2, _free_port(), k, 16, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        for gi in range(4):
            assert (tmp_path / ("x_rank%d_graph%d" % (rank, gi))).read_text() == "ok", (rank, gi)
    assert sum(int((tmp_path / ("x_rank%d_offers" % r)).read_text()) for r in range(2)) > 0


@pytest.mark.parametrize("k", [1, 10])
def test_thread_ranks_exchange_thresholds(lib, orc, k):
    """The same exchange with the ranks as threads of one process
    (ThreadGather, the way shards sharing one GPU context are driven): the
    merged top-k is the graph's and no shard scans more arcs than alone."""
    import threading

    import oracle
    from paper_1507_01490_gb300 import graphgen
    from paper_1507_01490_gb300.exchange import ThreadGather, ThresholdExchange
    orc.build()
    world = 2
    for g in [graphgen.ba(2000, 3, seed=1), graphgen.gnp(700, 0.006, seed=3, directed=True)]:
        order = oracle.order(g)
        if g.directed:
            _, al, om, _ = oracle.alpha_omega(g)
            bounds = (al, om)
        else:
            _, rr = oracle.farness_all(g)
            bounds = (rr, rr)
        tg = ThreadGather(world)
        res, errs, offers = [None] * world, [], [0] * world

        def rank_main(rank):
            try:
                src = order[B.shard_positions(g.n, rank, world)]
                alone = oracle.ShardRun(g, k, src, bounds)
                alone.step(len(src) + 1)
                run = oracle.ShardRun(g, k, src, bounds)
                ex = ThresholdExchange(period_s=0, gather=tg.for_rank(rank))
                ex.run(run.key, run.offer, lambda: run.step(16))
                offers[rank] = ex.offers
                res[rank] = run.result()
                assert res[rank][3]["m_vis"] <= alone.result()[3]["m_vis"]
            except BaseException as e:   # reported by the main thread
                errs.append(e)
                tg.bar.abort()

        ts = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errs, errs
        mi, mf, mr = B.bcm_topk_merge(np.concatenate([x[0] for x in res]), np.concatenate([x[1] for x in res]),
                                      np.concatenate([x[2] for x in res]), k)
        fa, ra = oracle.farness_all(g)
        exp = oracle.topk(fa, ra, k)
        assert np.array_equal(mi, exp) and np.array_equal(mf, fa[exp]) and np.array_equal(mr, ra[exp]), g.name
