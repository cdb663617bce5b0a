"""Pins the oracle's top-k selection: exact rational ranking, ties by id."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _brute_rank(f, r):
    def key(v):
        s = Fraction(0) if r[v] <= 1 else Fraction((int(r[v]) - 1) ** 2, int(f[v]))
        return (-s, v)
    return sorted(range(len(f)), key=key)


def test_golden_example(orc, gen):
    ex = json.load(open(os.path.join(GOLDEN, "topk_example.json")))
    e = np.array(ex["edges"])
    g = gen.csr_from_arcs(ex["n"], e[:, 0], e[:, 1], directed=False)
    f, r = orc.farness_all(g)
    assert f.tolist() == ex["farness"] and r.tolist() == ex["reach"]
    assert orc.topk(f, r, ex["n"]).tolist() == ex["ranking"]
    assert orc.topk(f, r, 3).tolist() == ex["ranking"][:3]
    assert orc.topk(f, r, 50).tolist() == ex["ranking"]


@pytest.mark.parametrize("seed", range(25))
def test_random_keys_with_ties(orc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    r = rng.integers(1, 6, n).astype(np.uint32)
    f = np.where(r > 1, rng.integers(1, 12, n) * (r - 1), 0).astype(np.uint64)
    k = int(rng.integers(1, n + 3))
    assert orc.topk(f, r, k).tolist() == _brute_rank(f, r)[:k]


def test_large_values_exact(orc):
    # keys that differ only beyond double precision: (r-1)^2/f with r ~ 2^30
    r = np.array([2**30, 2**30, 2**30 - 1], np.uint32)
    f = np.array([2**40 + 1, 2**40, 2**40 - 2**11], np.uint64)
    assert orc.topk(f, r, 3).tolist() == _brute_rank(f, r)


@pytest.mark.parametrize("g_name", ["cycle", "complete", "dcycle"])
def test_vertex_transitive_all_tied(orc, gen, g_name):
    g = getattr(gen, g_name)(17)
    ids, f, r = orc.topk_exhaustive(g, 5)
    assert ids.tolist() == [0, 1, 2, 3, 4]
    assert len(set(f.tolist())) == 1


def test_k_zero_and_empty(orc):
    assert orc.topk(np.zeros(0, np.uint64), np.zeros(0, np.uint32), 4).size == 0
    assert orc.topk(np.array([3], np.uint64), np.array([2], np.uint32), 0).size == 0


def test_processing_order(orc, gen):
    g = gen.star(6)
    assert orc.order(g).tolist() == [0, 1, 2, 3, 4, 5]
    g = gen.path(5)          # degrees 1,2,2,2,1
    assert orc.order(g).tolist() == [1, 2, 3, 0, 4]
    g = gen.disjoint_union(gen.path(2), gen.star(4), gen.empty(1))   # degrees 1,1,3,1,1,1,0
    assert orc.order(g).tolist() == [2, 0, 1, 3, 4, 5, 6]
