"""Sharding of independent canonical solves across ranks (one GPU per rank).

Independent Hamiltonians need no exchange: each rank solves its own share of a
batch and only scalars are reduced for timing. The share is chosen by the
longest-processing-time rule on the solve cost, which grows as N^3 (every
product of the recursion is an N x N x N GEMM).
"""
from __future__ import annotations

from typing import List, Sequence


def lpt_partition(weights: Sequence[float], parts: int) -> List[List[int]]:
    """Indices of `weights` split into `parts` lists by the LPT rule: items in
    decreasing weight, each to the currently lightest part (ties to the lowest
    part index). Every index appears exactly once; each list is returned in
    increasing index order. The heaviest part is at most 4/3 - 1/(3 parts) of
    the optimum (Graham's bound)."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    loads = [0.0] * parts
    out: List[List[int]] = [[] for _ in range(parts)]
    for i in order:
        p = min(range(parts), key=lambda q: (loads[q], q))
        out[p].append(i)
        loads[p] += float(weights[i])
    return [sorted(o) for o in out]


def cube_weights(sizes: Sequence[int]) -> List[float]:
    """Solve-cost weights of systems of the given sizes (N^3)."""
    return [float(n) ** 3 for n in sizes]
