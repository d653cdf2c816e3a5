"""Sharding a population of robots over GPUs (one process per GPU).

Robots are independent units: no step of the simulation exchanges data
between them, so a population splits into per-GPU shards that each rank
simulates with its own simulator context, and the only communication is the
gather of the per-robot results (fitness, 4 bytes each) to the host.  The
paper notes that evolutionary workloads need very little communication
between machines (Sec. 7) and allocates variants between devices in
proportion to their measured speed (Sec. 6); here the devices are identical
GPUs, so shards are balanced by a per-robot cost model instead.

Cost model: a robot's step cost grows about quadratically with its bodies
(mass matrix, Cholesky and the box/box pair count are all O(nb^2)), the same
estimate the simulator uses to order its first launch.

The gather runs over a gloo process group on host tensors, whatever backend
the default group uses, so it needs no GPU collective.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from . import population as P


def predicted_cost(pop: P.Population) -> np.ndarray:
    """Relative per-step cost of every robot (bodies squared)."""
    nb = np.asarray(pop.nb, dtype=np.float64)
    return nb * nb


def balanced_shards(cost: Sequence[float], world: int) -> list[np.ndarray]:
    """Split robots 0..n-1 into `world` contiguous shards of about equal cost.

    Shard r holds the robots whose cumulative cost midpoint falls in
    [r T / world, (r + 1) T / world), with T the total cost, so no shard
    exceeds its share by more than one robot's cost.  Every robot is in
    exactly one shard; shards are empty only when there are fewer robots
    than ranks.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    c = np.asarray(cost, dtype=np.float64)
    if c.ndim != 1 or np.any(c < 0) or not np.all(np.isfinite(c)):
        raise ValueError("cost must be a finite, non-negative 1-d array")
    n = c.size
    if n == 0:
        return [np.zeros(0, np.int64) for _ in range(world)]
    total = c.sum()
    if total <= 0:
        mid = (np.arange(n) + 0.5) / n
    else:
        mid = (np.cumsum(c) - 0.5 * c) / total
    owner = np.minimum((mid * world).astype(np.int64), world - 1)
    if n < world:
        return [np.flatnonzero(owner == r) for r in range(world)]
    # shard r starts at its first owned robot, moved so that every shard
    # keeps at least one robot
    starts = np.searchsorted(owner, np.arange(world), side="left")
    for r in range(world):
        lo = 0 if r == 0 else starts[r - 1] + 1
        starts[r] = min(max(starts[r], lo), n - world + r)
    bounds = np.append(starts, n)
    return [np.arange(bounds[r], bounds[r + 1]) for r in range(world)]


def _gloo_group(dist):
    """A gloo group over all ranks (the default group when it already is gloo)."""
    if dist.get_backend() == "gloo":
        return None
    return dist.new_group(backend="gloo")


def run_sharded(pop: P.Population, simulate: Callable[[P.Population], np.ndarray], dist=None,
                cost: Sequence[float] | None = None) -> np.ndarray:
    """Simulate this rank's shard and return the results of all robots, in
    population order, on every rank.

    simulate(shard_population) -> per-robot float array.  With `dist` None or
    a single rank the whole population is simulated locally.
    """
    world = dist.get_world_size() if dist is not None else 1
    if world <= 1:
        return np.asarray(simulate(pop), dtype=np.float64)
    rank = dist.get_rank()
    shards = balanced_shards(predicted_cost(pop) if cost is None else cost, world)
    mine = shards[rank]
    local = np.asarray(simulate(pop.subset(mine)), dtype=np.float64) if mine.size else np.zeros(0)
    if local.shape != (mine.size,):
        raise ValueError(f"simulate returned shape {local.shape} for a shard of {mine.size} robots")
    group = _gloo_group(dist)
    parts: list = [None] * world
    dist.all_gather_object(parts, local, group=group)
    out = np.empty(pop.n, dtype=np.float64)
    for r in range(world):
        if parts[r].shape != (shards[r].size,):
            raise RuntimeError(f"rank {r} returned {parts[r].shape} results for {shards[r].size} robots")
        out[shards[r]] = parts[r]
    return out
