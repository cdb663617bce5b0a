"""Per-graph tuning of the launch parameters by measurement.

The result of bcm_topk does not depend on these parameters (every choice
returns the same ids, farness and reach; this module checks that on every
trial); only the time does.  So each graph gets the setting that ran
fastest on it:

  lanes        sources per per-CTA wave (64, 128, 256)
  grid_lanes   sources per grid-wide wave (64, 128, 256)
  pull_div     the push/pull switch: a grid level is pulled once its
               frontier's out-arcs reach n*W/pull_div
  threads      the per-CTA kernel's block shape (256, 512, 1024 threads)
  per_cta      which per-CTA kernel runs after the grid-wide waves: the
               library's choice, bit-lane waves (BCM_NO_SPARSE) or one
               source per CTA (BCM_SPARSE); tried on graphs whose largest
               degree is at most 64, where the two are close

Search: coordinate descent from the library defaults -- one parameter at a
time over its candidates with the others held, kept if it beats the best
by more than the noise margin -- for a fixed number of rounds.  Each trial
is the median device time (CUDA events, bcm_stats.kernel_ms) of a few runs
after a warm-up.  Results are cached in a JSON file keyed by the graph's
content hash, k, and the GPU's name.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import bcm

SPACE = {
    "grid_lanes": (128, 64, 256),
    "pull_div": (32, 8, 16, 64, 128),
    "lanes": (64, 128, 256),
    "threads": (512, 256, 1024),
}
DEFAULTS = {"grid_lanes": 128, "pull_div": 32, "lanes": 64, "threads": 512}
PER_CTA = {"auto": 0, "bitlanes": bcm.BCM_NO_SPARSE, "sparse": bcm.BCM_SPARSE}
KERNEL_MAX_DEG = 64   # graphs with a larger degree keep the library's choice
KERNEL_TRIAL_MS = 200.0   # ... and so do graphs whose default run takes longer


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:
        return "unknown"


def _valid(cfg) -> bool:
    return cfg["threads"] >= cfg["lanes"]


def options_of(cfg):
    """bcm_topk keyword arguments of a tuned setting."""
    kw = dict(cfg)
    per = kw.pop("per_cta", "auto")
    return kw, PER_CTA[per]


def measure(h, k, cfg, reps=3, flags=0):
    """Median kernel time (ms) of bcm_topk with cfg, and its result."""
    kw, extra = options_of(cfg)
    flags = flags | extra
    h.topk(k, flags=flags, **kw)
    ts = []
    res = None
    for _ in range(reps):
        ids, far, reach, st = h.topk(k, flags=flags, **kw)
        ts.append(st["kernel_ms"])
        res = (ids, far, reach)
    return float(np.median(ts)), res


def tune(h, k=10, rounds=2, reps=3, margin=0.02, flags=0, log=None, kernels=False):
    """Coordinate descent over SPACE (and, with kernels, the per-CTA kernel)
    on the handle `h` (a BcmGraph).  Returns (best config, its time in ms,
    trials)."""
    best = dict(DEFAULTS)
    space = dict(SPACE)
    if kernels:
        best["per_cta"] = "auto"
    best_t, ref = measure(h, k, best, reps, flags)
    # the other kernel can be far slower on a graph that suits the default
    # (bit lanes on a large lattice: a hundred times), so it is tried only
    # where a trial is cheap
    if kernels and best_t <= KERNEL_TRIAL_MS:
        space["per_cta"] = tuple(PER_CTA)
    trials = [(dict(best), best_t)]
    for _ in range(rounds):
        changed = False
        for name, values in space.items():
            for v in values:
                if v == best[name]:
                    continue
                cfg = dict(best)
                cfg[name] = v
                if not _valid(cfg):
                    continue
                t, res = measure(h, k, cfg, reps, flags)
                trials.append((dict(cfg), t))
                if not all(np.array_equal(a, b) for a, b in zip(ref, res)):
                    raise RuntimeError("autotune: result changed with %r" % (cfg,))
                if log:
                    log("  %s -> %.3f ms" % (cfg, t))
                if t < best_t * (1.0 - margin):
                    best, best_t, changed = cfg, t, True
        if not changed:
            break
    return best, best_t, trials


class Cache:
    """Tuned settings on disk, keyed by graph hash, k and device."""

    def __init__(self, path: str):
        self.path = path
        self.data = {}
        if os.path.exists(path):
            try:
                self.data = json.load(open(path))
            except (OSError, ValueError):
                self.data = {}

    @staticmethod
    def key(graph_hash: str, k: int) -> str:
        return "%s|k=%d|%s" % (graph_hash, k, _device_name())

    def get(self, graph_hash, k):
        return self.data.get(self.key(graph_hash, k))

    def put(self, graph_hash, k, cfg, ms):
        self.data[self.key(graph_hash, k)] = {"config": cfg, "kernel_ms": ms, "when": time.time()}
        tmp = self.path + ".tmp%d" % os.getpid()
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tuned_options(h, graph, k=10, cache_path=None, **kw):
    """The cached setting for (graph, k), tuning it first if needed.
    Returns (config dict, seconds spent tuning, whether it came from the cache)."""
    gh = graph.hash64()
    cache = Cache(cache_path) if cache_path else None
    if cache:
        hit = cache.get(gh, k)
        if hit:
            return hit["config"], 0.0, True
    t0 = time.perf_counter()
    kw.setdefault("kernels", bool(graph.n) and int(graph.degrees().max()) <= KERNEL_MAX_DEG)
    cfg, ms, _ = tune(h, k, **kw)
    spent = time.perf_counter() - t0
    if cache:
        cache.put(gh, k, cfg, ms)
    return cfg, spent, False
