"""Seeded synthetic tight-binding inputs shared by the oracle, the tests and the bench.

This module builds Hamiltonians only. It holds none of the density-matrix
arithmetic: no Fermi function, no recursion, no response. Both the CPU oracle
and the CUDA path receive the same FP64 arrays from here.
"""
from .tightbinding import (  # noqa: F401
    Problem,
    chain_1d,
    cubic_lattice,
    banded_random,
    cluster_sizes,
    nonorthogonal_cluster,
    clusters,
    workload,
    WORKLOADS,
)
