"""GB300 (sm_103a) incremental dynamic community detection with Delta-screening.

Hot path (hand-written CUDA in ``csrc/``, behind the C ABI of ``include/dcd.h``):
batch sort-merge into CSR, Delta-screening of the batch (Algorithm 2 of
arXiv 1904.08553), degree-binned Louvain local moving over R_t, and graph
compaction.  ``dcd`` is the ctypes binding; ``synth`` the seeded workload
generators.
"""

__all__ = ["dcd", "synth"]
