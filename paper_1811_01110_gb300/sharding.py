"""Multi-GPU partition of one evaluation: targets are independent (each target
belongs to exactly one center and one group), so an evaluation splits into
per-rank target shards with no exchange; the outputs are concatenated."""
import numpy as np


def shard_targets(geometry, world_size):
    """Split the targets into `world_size` shards of near-equal pair count.

    Targets are ordered by group (so a group's targets, which share one source
    list, stay together where possible) and cut at cumulative pair-count
    quantiles.  Returns a list of sorted int64 index arrays covering every
    target exactly once."""
    g = geometry
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    per_group = g.group_source_counts()
    tg = np.asarray(g.ctr_group)[np.asarray(g.tgt_center)]
    order = np.argsort(tg, kind="stable")
    cost = per_group[tg[order]].astype(np.float64) + 1.0
    csum = np.cumsum(cost)
    total = csum[-1] if len(csum) else 0.0
    cuts = [0]
    for r in range(1, world_size):
        cuts.append(int(np.searchsorted(csum, total * r / world_size)))
    cuts.append(len(order))
    return [np.sort(order[cuts[r]:cuts[r + 1]]).astype(np.int64) for r in range(world_size)]


def gather_outputs(parts, shards, n_tgt, dtype=np.float64):
    """Place per-rank outputs (in shard order) back into one target-indexed array."""
    out = np.zeros(n_tgt, dtype=dtype)
    for part, idx in zip(parts, shards):
        out[idx] = part
    return out
