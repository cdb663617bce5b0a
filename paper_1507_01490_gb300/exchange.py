"""Threshold exchange between the shards of one graph (one rank per GPU).

Section 2's parallel version keeps a single x_k, the current k-th best
closeness, for all threads.  With the sources sharded over ranks
(``bcm_options.shard_*``), each rank's run only knows its own shard's k-th key.
The exchange shares them while the runs go on: every round each rank reads its
run's published key (``bcm_topk_threshold``), one all-gather over a CPU
(gloo) group brings every rank's key and "finished" flag to all ranks, and
each rank offers the best key to its own run (``bcm_topk_offer``), which cuts
with it from its next level on.

Any shard's k-th key is a valid threshold for every shard: at least k
vertices of the graph rank at or before it.  So the exchange never changes
the merged top-k; it only lets a shard stop sources earlier.  It runs on the
host between kernel levels and needs no collective inside a kernel.  The
rounds end in the same round on every rank: once all ranks report finished.

Keys are (valid, N, F, id) with N = (r-1)^2, F = f, as in ``bcm_key``; both
stay below 2^62, so they travel as int64.
"""
from __future__ import annotations

import threading
import time

NO_KEY = (0, 0, 1, 0)


def key_before(a, b) -> bool:
    """Key a = (valid, N, F, id) ranks strictly before key b; an invalid key
    ranks after every valid one."""
    if not a[0]:
        return False
    if not b[0]:
        return True
    l, r = a[1] * b[2], b[1] * a[2]
    if l != r:
        return l > r
    return a[3] < b[3]


def best_key(keys):
    best = NO_KEY
    for k in keys:
        if key_before(k, best):
            best = tuple(int(x) for x in k)
    return best


class ThreadGather:
    """All-gather among `world` threads of one process: shards of one graph
    run from threads that share one GPU context (and its streams), as the
    serving loop runs several graphs.  for_rank(r) is rank r's gather."""

    def __init__(self, world: int, timeout_s: float = 60.0):
        self.rows = [None] * world
        self.bar = threading.Barrier(world, timeout=timeout_s)

    def for_rank(self, rank: int):
        def gather(row):
            self.rows[rank] = tuple(int(x) for x in row)
            self.bar.wait()
            out = list(self.rows)
            self.bar.wait()           # every rank has read the round's rows
            return out
        return gather


class ThresholdExchange:
    """Rounds of key exchange among the ranks of `group` (a gloo process
    group; None = the default group), or through `gather` (row -> every
    rank's row, e.g. ThreadGather.for_rank).  period_s: pause between rounds."""

    def __init__(self, group=None, period_s: float = 2e-4, gather=None):
        self.group = group
        self.period_s = period_s
        self.gather = gather
        self.rounds = 0
        self.offers = 0

    def _all_gather(self, row):
        if self.gather is not None:
            return self.gather(row)
        import torch
        import torch.distributed as dist
        world = dist.get_world_size(self.group)
        t = torch.tensor(row, dtype=torch.int64)
        out = [torch.zeros(len(row), dtype=torch.int64) for _ in range(world)]
        dist.all_gather(out, t, group=self.group)
        return [tuple(int(x) for x in o.tolist()) for o in out]

    def run(self, read_key, offer_key, poll):
        """Exchange until every rank's run has finished.

        poll()        -> True once this rank's run has finished (it may also
                         advance the run, for a run driven from the host);
        read_key()    -> this rank's current k-th key (valid, N, F, id);
        offer_key(k)  -> gives key k to this rank's run (only while it runs).
        Returns the best key seen."""
        done = False
        offered = NO_KEY
        best = NO_KEY
        while True:
            if not done:
                done = bool(poll())
            mine = tuple(int(x) for x in read_key())
            out = self._all_gather([int(done), *mine])
            self.rounds += 1
            keys = [tuple(o[1:]) for o in out]
            best = best_key(keys + [best])
            if not done and key_before(best, mine) and key_before(best, offered):
                offer_key(best)
                offered = best
                self.offers += 1
            if all(int(o[0]) for o in out):
                return best
            if self.period_s:
                time.sleep(self.period_s)
