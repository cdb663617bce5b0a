"""Writes the full-size top-k goldens: the exact top-k of a named workload as
the oracle's sequential Algorithm 1 (BCM with BFSCut, Sections 2.1-2.3)
returns it.  This script calls only the oracle and the seeded input
generators; no value in the files it writes comes from the CUDA library.

Algorithm 1 reaches exactly the textbook top-k (one BFS per vertex, ties by
smaller id), and the oracle's implementation is pinned against the
exhaustive definition on many small graphs (tests/test_oracle_bcm.py), so
these files are the complete answer, not a sample: every vertex of the graph
was either run to the end of its BFS or stopped by a bound that proves it
ranks below the k-th entry.

Usage (minutes of CPU per workload and k; the R-MAT runs are the long ones):
    python tests/golden/make_fullsize.py chunglu1m 1 10 100
    python tests/golden/make_fullsize.py rmat20 10

Each (workload, k) goes to tests/golden/fullsize_<workload>_k<k>.json with
the graph's content hash, so a test can tell that it runs on the same graph.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1507_01490_gb300 import graphgen  # noqa: E402  (inputs only)


def golden_path(name: str, k: int) -> str:
    return os.path.join(HERE, "fullsize_%s_k%d.json" % (name, k))


def main(argv):
    if len(argv) < 2:
        print(__doc__)
        return 2
    name = argv[0]
    ks = [int(a) for a in argv[1:]]
    g = graphgen.workload(name)
    h = g.hash64()
    for k in ks:
        t0 = time.time()
        # digraphs: alpha/omega with Section 2.3's biggest-SCC refinement (the
        # top-k is the same with either form of the bounds; this one cuts more)
        ids, far, reach, st = oracle.bcm(g, k, refined=g.directed)
        sec = time.time() - t0
        rec = {
            "workload": name,
            "graph": g.name,
            "n": g.n,
            "m": g.m,
            "directed": bool(g.directed),
            "csr_sha256_16": h,
            "k": k,
            "ids": [int(x) for x in ids],
            "farness": [int(x) for x in far],
            "reach": [int(x) for x in reach],
            "oracle_stats": {kk: int(v) for kk, v in st.items()},
            "oracle_seconds": round(sec, 1),
            "source": "oracle.bcm (sequential Algorithm 1 with BFSCut), tests/golden/make_fullsize.py",
        }
        with open(golden_path(name, k), "w") as fh:
            json.dump(rec, fh, indent=1)
            fh.write("\n")
        print("%s k=%d: %d entries, m_vis %d, %.1f s" % (name, k, len(ids), st["m_vis"], sec), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
