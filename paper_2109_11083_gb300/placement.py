"""Placement of independent systems onto GPUs (host logic, no collective).

Boxes of a batch or requests of a served stream share nothing, so a run over
several GPUs only decides which GPU holds which system; results are gathered
on the host.  Every rank computes the same assignment from the same inputs.
"""
from __future__ import annotations


def assign(sizes, world: int) -> list[int]:
    """Owner rank of each system: largest first to the least loaded rank
    (ties to the lower rank index), load = summed particle count."""
    order = sorted(range(len(sizes)), key=lambda k: (-sizes[k], k))
    load = [0] * world
    owner = [0] * len(sizes)
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += sizes[k]
    return owner


def shard_systems(specs, rank: int, world: int):
    """The systems (dicts with a particle count "n") that `rank` of `world`
    ranks holds."""
    owner = assign([s["n"] for s in specs], world)
    return [specs[k] for k in range(len(specs)) if owner[k] == rank]


def least_loaded(loads) -> int:
    """The GPU a newly admitted system goes to: the one with the fewest
    resident particles (ties to the lower index)."""
    return min(range(len(loads)), key=lambda q: (loads[q], q))
