"""Multi-GPU partition of one evaluation: targets are independent (each target
belongs to exactly one center and one group), so an evaluation splits into
per-rank target shards with no exchange; the outputs are concatenated.

Sources, centers and pair lists are replicated on every rank; each rank's
plan holds only its own targets (`shard_geometry`).  `distributed_eval`
runs one evaluation over a torch.distributed group: every rank evaluates its
shard and one all-gather per layer of the (padded) output tensors
reassembles them -- device tensors under NCCL, host tensors under gloo."""
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


def _as_real_tensor(torch, v, device):
    """v (numpy array or torch tensor) as a real torch tensor on `device`:
    complex values become a trailing (re, im) axis."""
    t = v if isinstance(v, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(v))
    t = t.to(device)
    return torch.view_as_real(t) if t.is_complex() else t


def distributed_eval(geometry, evaluate, rank, world_size, all_gather=None, device=None):
    """One evaluation split over `world_size` ranks with no data-path exchange.

    evaluate(shard) -> {layer: 1-D array over the shard's targets} runs this
    rank's part (a Plan on this rank's GPU); its values may be numpy arrays or
    torch tensors, host or device.  The shards' outputs are then exchanged by
    one all-gather per layer of tensors padded to the longest shard (every
    rank knows every shard's size, so no size exchange is needed).
    all_gather has the contract of torch.distributed.all_gather(tensor_list,
    tensor) and defaults to it; device is where the gathered tensors live:
    the outputs' own device under NCCL (the data plane then stays on the
    GPUs), the host under gloo (the default for any other backend).  Every
    rank returns the full {layer: array over all targets}, as numpy arrays
    if evaluate returned numpy arrays, else as torch tensors on `device`."""
    import torch
    import torch.distributed as dist
    shards = shard_targets(geometry, world_size)
    mine = evaluate(shard_geometry(geometry, shards[rank]))
    as_numpy = not any(isinstance(v, torch.Tensor) for v in mine.values())
    if device is None:
        on_nccl = all_gather is None and dist.is_initialized() and dist.get_backend() == "nccl"
        dev_of = [v.device for v in mine.values() if isinstance(v, torch.Tensor) and v.is_cuda]
        device = dev_of[0] if (on_nccl and dev_of) else torch.device("cpu")
    gather = all_gather or dist.all_gather
    n_max = max(len(s) for s in shards)
    n_tgt = int(np.asarray(geometry.tgt_center).shape[0])
    result = {}
    for layer in sorted(mine):
        part = _as_real_tensor(torch, mine[layer], device)
        padded = torch.zeros((n_max,) + tuple(part.shape[1:]), dtype=part.dtype, device=device)
        padded[: part.shape[0]] = part
        parts = [torch.empty_like(padded) for _ in range(world_size)]
        gather(parts, padded)
        full = torch.zeros((n_tgt,) + tuple(part.shape[1:]), dtype=part.dtype, device=device)
        for r, idx in enumerate(shards):
            if len(idx):
                full[torch.from_numpy(idx).to(device)] = parts[r][: len(idx)]
        if full.dim() == 2:                              # complex values
            full = torch.view_as_complex(full.contiguous())
        result[layer] = full.cpu().numpy() if as_numpy else full
    return result
