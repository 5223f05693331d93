"""Partition of one batch of stacks across ranks by estimated cost.

Stacks are independent units of the batched likelihood (no data moves
between them), so several GPUs can split one batch: each rank evaluates a
subset of the stacks against a replica of the datasets.  The cost of a stack
is proportional to its evaluations times its interfaces,
(n + 1) x N_Q x K, since the layer recursion and its adjoint run once per
interface for every (Q point, quadrature node) pair.  The partition is the
longest-processing-time-first greedy: stacks in decreasing cost, each to the
rank with the least assigned cost so far (ties to the lower rank), which
keeps the largest load within 4/3 of the optimum.  Host logic only.
"""
from __future__ import annotations

import numpy as np


def stack_costs(n_layers, q_len, n_quad: int) -> np.ndarray:
    """(n + 1) x N_Q x K per stack, as float64."""
    n = np.asarray(n_layers, np.float64)
    m = np.asarray(q_len, np.float64)
    return (n + 1.0) * m * float(n_quad)


def cost_partition(costs, world: int) -> list[np.ndarray]:
    """Indices of the stacks each of `world` ranks evaluates (ascending
    within a rank); every stack appears in exactly one rank's list."""
    costs = np.asarray(costs, np.float64)
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    owner = np.empty(costs.size, np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return [np.flatnonzero(owner == r) for r in range(world)]


def workload_partition(wl, world: int) -> list[np.ndarray]:
    """cost_partition of a workload's stacks (workloads.Workload)."""
    q_len = (wl.q_off[1:] - wl.q_off[:-1])[wl.dataset]
    return cost_partition(stack_costs(wl.n_layers, q_len, wl.n_quad), world)
