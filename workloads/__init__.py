"""Seeded synthetic workloads for the consensus-clustering sweep.

This package only makes inputs: graphs in CSR form and input partitions of
their vertices.  It holds none of the consensus method's arithmetic, so both
the CUDA path and the CPU oracle can be fed from it without sharing logic.

* ``graphs``      planted-partition SBM, LFR-style power-law graphs and
                  Gaussian-mixture kNN graphs, all returned as
                  (row_off int64[n+1], col int32[nnz], truth int32[n]).
* ``partitions``  the merge / split / neighbour-relabel perturbation that turns
                  planted labels into k input partitions.
* ``configs``     the named workloads (sizes and parameters of each).
"""
from .graphs import csr_from_edges, sbm, lfr_like, knn_mixture  # noqa: F401
from .partitions import perturb, perturb_many  # noqa: F401
from .configs import make_config, CONFIG_NAMES  # noqa: F401
