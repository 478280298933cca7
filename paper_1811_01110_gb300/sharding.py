"""Multi-GPU partition of one evaluation: targets are independent (each target
belongs to exactly one center and one group), so an evaluation splits into
per-rank target shards with no exchange; the outputs are concatenated.

Sources, centers and pair lists are replicated on every rank; each rank's
plan holds only its own targets (`shard_geometry`).  `distributed_eval`
runs one evaluation over a torch.distributed group: every rank evaluates its
shard and one all-gather of the outputs reassembles them."""
import types

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


def shard_geometry(geometry, idx):
    """The geometry restricted to the targets `idx` (sorted int64): sources,
    centers, groups and pair lists are kept as they are; target positions,
    centers and normals are subset.  Works on any object carrying the
    library's geometry fields."""
    g = geometry
    idx = np.asarray(idx, dtype=np.int64)
    tn = getattr(g, "tgt_normal", None)
    fields = {name: getattr(g, name) for name in ("src_xyz", "src_weight", "src_normal", "ctr_xyz",
                                                  "ctr_group", "group_range_start", "range_begin",
                                                  "range_end")}
    fields["ctr_radius"] = getattr(g, "ctr_radius", None)
    fields["tgt_xyz"] = np.ascontiguousarray(np.asarray(g.tgt_xyz)[:, idx])
    fields["tgt_center"] = np.ascontiguousarray(np.asarray(g.tgt_center)[idx])
    fields["tgt_normal"] = None if tn is None else np.ascontiguousarray(np.asarray(tn)[:, idx])
    return types.SimpleNamespace(**fields)


def distributed_eval(geometry, evaluate, rank, world_size, all_gather_object):
    """One evaluation split over `world_size` ranks with no data-path exchange.

    evaluate(shard) -> {layer: 1-D array over the shard's targets} runs this
    rank's part (a Plan on this rank's GPU); all_gather_object is
    torch.distributed.all_gather_object (or any function with its contract).
    Every rank returns the full {layer: array over all targets}."""
    shards = shard_targets(geometry, world_size)
    mine = evaluate(shard_geometry(geometry, shards[rank]))
    mine = {k: np.asarray(v) for k, v in mine.items()}
    parts = [None] * world_size
    all_gather_object(parts, mine)
    n_tgt = int(np.asarray(geometry.tgt_center).shape[0])
    return {k: gather_outputs([p_[k] for p_ in parts], shards, n_tgt, dtype=mine[k].dtype)
            for k in mine}
