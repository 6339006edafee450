"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle scripts.

This package only produces inputs (graphs in in-CSR form, source nodes, diagonal
vectors, sample-count vectors).  It contains none of the SimRank arithmetic: the
oracle and the CUDA library each compute the method on their own.
"""
from .graphs import (  # noqa: F401
    edges_to_in_csr,
    erdos_renyi,
    chung_lu,
    rmat,
    rmat_torch,
    chung_lu_torch,
    random_sources,
    uniform_diagonal,
    out_star,
    in_star,
    directed_cycle,
    complete_digraph,
    two_parents,
    random_small,
    with_dangling,
)
