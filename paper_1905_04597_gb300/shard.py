"""Split of independent lattice instances across ranks (one process per GPU).

The instances of a batch are independent problems: nothing is exchanged
between them, so a multi-GPU run gives each rank a share of the instances and
no data-path collective. Shares are balanced by population bytes, the
quantity a bandwidth-bound step's time follows.
"""
from __future__ import annotations


def instance_bytes(cfg: dict, elem: int = 4) -> int:
    """Population bytes of one 2D instance per buffer: Q nx ny elem, Q the
    product of the two axes' velocity counts (2N+1, or 2N+2 on an axis of the
    2N+2 hierarchy; D1Q3 along x when x_level is 1)."""
    N = cfg["k"] + 1
    NX = cfg.get("x_level") or N
    zv = cfg.get("zv_axes", 0)
    qy = 2 * N + 1 + (1 if zv & 2 else 0)
    qx = 2 * NX + 1 + (1 if zv & 1 else 0)
    return qx * qy * cfg["nx"] * cfg["ny"] * elem


def partition_by_bytes(sizes, world: int) -> list[list[int]]:
    """Greedy longest-first split of instances of the given sizes into `world`
    shares: in order of decreasing size (ties by index), each instance goes to
    the share with the fewest bytes so far (ties to the lowest rank). Returns
    the instance indices of each rank, ascending. Deterministic, so every rank
    computes the same split without communicating; the largest share exceeds
    the mean by less than the largest instance."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]
