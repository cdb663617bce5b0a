"""Exact top-k closeness centrality (Borassi, Crescenzi, Marino, arXiv
1507.01490) on one GB300: BFSCut run as multi-source bitset BFS waves in
hand-written sm_103a CUDA, behind the C-ABI of include/bcm.h.

``bcm``       the Python binding of that C-ABI (same function names).
``graphgen``  seeded synthetic graphs (inputs only).
``serve``     a continuous-batching request loop over the C-ABI.
"""
from .bcm import BcmError, BcmGraph  # noqa: F401
