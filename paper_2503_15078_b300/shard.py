"""Sharding a batch of independent scenes over the ranks of a job (one GPU per rank).

Scenes of a batch share no element, no contact and no unknown, so a batch splits by scene
with no exchange between the ranks: every rank simulates its own scenes in one simulator
(sim_create_batch) and nothing crosses ranks on the data path. The cost of a scene's
local-global iteration is dominated by the two profile products, which read the scene's
nnz(S~) values each (Sec. 4.2, Theorem 1: the rows of the sparse inverse), so the scenes are
balanced by nnz(S~) with the longest-processing-time rule: scenes in decreasing cost, each to
the rank with the smallest total so far (ties: the lower scene index first, the lower rank).
Every rank computes the same partition from the same inputs, so no rank has to send it.
"""
from __future__ import annotations

from typing import List, Sequence


def partition(costs: Sequence[float], world: int) -> List[List[int]]:
    """Scene indices of each rank (ascending within a rank) from per-scene costs.

    The largest total is at most 4/3 of the best possible split plus nothing more than the
    largest single cost (the rule's bound); every scene goes to exactly one rank."""
    if world < 1:
        raise ValueError("world must be at least 1")
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def scene_costs(scenes, h=None) -> List[int]:
    """nnz(S~) of every scene from the host precompute (the product bytes per iteration are
    proportional to it)."""
    from . import Plan
    return [int(Plan(sc, h=h).info()["nnz_S"]) for sc in scenes]


def shard(scenes, rank: int, world: int, costs=None):
    """(indices, scenes) of this rank's part of the batch."""
    if not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    costs = scene_costs(scenes) if costs is None else costs
    idx = partition(costs, world)[rank]
    return idx, [scenes[i] for i in idx]
