"""Seeded synthetic inputs for APEX enumeration: library shapes, synthon embeddings,
random-init head weights and query descriptors.

This package holds no arithmetic of the method itself (no head evaluation, no
factorization, no selection). It is the one module shared by the FP64 oracle
(``oracle/``), the CUDA path (``paper_2510_24380_b300``), the tests and the
benchmark: both sides receive byte-identical inputs from it and nothing else.
"""
from .library import (
    CSL,
    Head,
    make_library,
    make_head,
    lognormal_slot_sizes,
    library_from_sizes,
)
from .configs import WORKLOADS, build_workload, subset_prefix, workload_sizes
from .queries import Query, query_single, queries_batched, queries_step, random_query, serving_stream, load_stats

__all__ = [
    "CSL", "Head", "make_library", "make_head", "lognormal_slot_sizes", "library_from_sizes",
    "WORKLOADS", "build_workload", "subset_prefix", "workload_sizes",
    "Query", "query_single", "queries_batched", "queries_step", "random_query", "serving_stream", "load_stats",
]
