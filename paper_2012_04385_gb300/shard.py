"""Sharding a batched ensemble of independent MR simulations by instance.

The instances of a batched run (the four-quadrant ensemble with uneven tree
depths) share nothing but the launches: every block id carries its instance
in bits 56..63 (Sec. 3's Morton ids with an instance prefix), the time step,
the conservation sums and the MR analysis are per instance.  Spreading the
instances over ranks (one process per GPU) therefore needs no data exchange
at all: each rank runs a batched context of its own instances, and only the
timings and per-instance results are gathered.  The paper distributes the
blocks of one simulation over MPI ranks with a level-wise space-filling curve
and halo messages; an ensemble needs none of that.

This module holds the host logic only: which instances a rank takes, the
rank's configuration, and the mapping of its local instance numbers back to
the ensemble's (for the seeded initial conditions).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .inputs import NB, RunConfig

MASK56 = np.uint64((1 << 56) - 1)


def instance_cost(cfg: RunConfig, inst: int) -> float:
    """Relative cost of an instance: its effective cell count (8^lmax times
    the base blocks), the bound its MR tree grows toward."""
    return float(np.prod(cfg.base_blocks)) * NB ** 3 * 8.0 ** cfg.lmax_of(inst)


def instance_shards(cfg: RunConfig, world: int) -> list[list[int]]:
    """Instances of each rank: greedy longest-processing-time assignment (the
    costliest instance first, to the least loaded rank; ties to the lower
    rank), each rank's list in ascending instance order.  Deterministic, so
    every rank computes the same partition without communicating."""
    if world < 1:
        raise ValueError("world < 1")
    order = sorted(range(cfg.n_instances), key=lambda i: (-instance_cost(cfg, i), i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += instance_cost(cfg, i)
    return [sorted(s) for s in out]


def shard_config(cfg: RunConfig, instances: list[int]) -> RunConfig:
    """The run configuration of a rank holding `instances` of the ensemble."""
    if not instances:
        raise ValueError("empty shard")
    return dataclasses.replace(cfg, n_instances=len(instances),
                               lmax=tuple(cfg.lmax_of(i) for i in instances),
                               name=f"{cfg.name}_shard")


def to_global_keys(keys, instances: list[int]) -> np.ndarray:
    """Block ids of a shard (local instance j in bits 56..63) with the
    ensemble's instance numbers instances[j] in their place."""
    keys = np.asarray(keys, dtype=np.uint64)
    loc = (keys >> np.uint64(56)).astype(np.int64)
    glob = np.asarray(instances, dtype=np.uint64)[loc]
    return (keys & MASK56) | (glob << np.uint64(56))


def shard_ic(ic, instances: list[int]):
    """An initial condition ic(cfg, geo, keys) of the ensemble, as seen by a
    shard: the shard's keys are mapped to the ensemble's instances first."""
    def f(cfg, geo, keys):
        return ic(cfg, geo, to_global_keys(keys, instances))
    return f
