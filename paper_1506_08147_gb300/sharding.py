"""Assignment of independent elements to ranks (one process per GPU).

Elements are independent units of ALB generation (Sec. II.B: inter-element
parallelism needs no communication), so a multi-GPU run splits the element
list with no collective on the data path.  The split is greedy
longest-processing-time by an estimated cost N_g * m^2 (the Gram and
Rayleigh-Ritz work per iteration grows with N_g m^2 and (3m)^3, the
former dominating at these sizes).
"""

from __future__ import annotations

import heapq


def element_cost(n, m: int) -> float:
    """Estimated relative cost of one element: N_g * m^2."""
    return float(n[0] * n[1] * n[2]) * float(m) * float(m)


def partition(costs, world: int):
    """Greedy LPT split of element indices into `world` lists (each sorted)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts = [[] for _ in range(world)]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def my_elements(descs, rank: int, world: int):
    """Indices of the elements rank `rank` solves."""
    costs = [element_cost(d["n"], d["m"]) for d in descs]
    return partition(costs, world)[rank]
