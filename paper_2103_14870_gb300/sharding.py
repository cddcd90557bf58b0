"""Assignment of independent meshes to ranks for the multi-GPU batch.

A batch of meshes has no coupling between meshes, so it shards across GPUs
with no collective on the data path: each rank steps the meshes assigned to
it as its own batch.  The assignment is the greedy longest-processing-time
rule: meshes in decreasing size (ties by index) each go to the rank with the
smallest load so far (ties by rank).  Every rank computes the same assignment
from the same sizes, so nothing is exchanged to agree on it.  The largest load
is at most 4/3 of the optimum (Graham's bound for this rule).
"""
from __future__ import annotations


def assign_meshes(sizes, world: int) -> list[list[int]]:
    """Mesh indices per rank (each list ascending) for `world` ranks; `sizes`
    are the per-mesh costs (for example tet counts)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = [int(s) for s in sizes]
    if any(s < 0 for s in sizes):
        raise ValueError("sizes must be >= 0")
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for k in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += sizes[k]
    return [sorted(x) for x in out]
