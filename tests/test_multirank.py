"""World-size-2 CPU (gloo) test of the sharded evaluation: each rank evaluates
its shard of targets, the outputs are all-gathered and reassembled, and the
result equals the single-rank evaluation exactly.  The per-rank evaluator is
the oracle here (no GPU); on GPUs it is a Plan over the rank's shard."""
import os
import socket

import numpy as np
import pytest

from paper_1811_01110_gb300.sharding import distributed_eval, gather_outputs, shard_geometry, shard_targets


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch.distributed as dist
    import oracle
    from tsqbx_inputs import configs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, mu, _ = configs.torus(24, 10)
    shards = shard_targets(g, world)
    mine = oracle.tsqbx_laplace(g, 7, mu, subset=shards[rank], slp=True, dlp=True)
    parts = [None] * world
    dist.all_gather_object(parts, {k: v.tolist() for k, v in mine.items()})
    if rank == 0:
        full = {k: gather_outputs([np.array(p[k]) for p in parts], shards, g.n_tgt)
                for k in ("slp", "dlp")}
        ref = oracle.tsqbx_laplace(g, 7, mu, slp=True, dlp=True)
        ok = all(np.array_equal(full[k], ref[k]) for k in ("slp", "dlp"))
        counts = [int(g.group_source_counts()[g.ctr_group[g.tgt_center[s]]].sum()) for s in shards]
        with open(result_path, "w") as f:
            f.write(f"{int(ok)} {counts[0]} {counts[1]}")
    # the package's driver, Helmholtz with all three layers on the oracle
    gh, muh, _ = configs.torus_helmholtz(16, 6, k=5.0)

    def evaluate(shard):
        return oracle.tsqbx_helmholtz(shard, 6, 5.0, muh, slp=True, dlp=True, sp=True)

    got = distributed_eval(gh, evaluate, rank, world)
    if rank == 0:
        ref = oracle.tsqbx_helmholtz(gh, 6, 5.0, muh, slp=True, dlp=True, sp=True)
        ok = all(np.array_equal(got[k], ref[k]) and got[k].dtype == np.complex128 for k in ref)
        with open(result_path, "a") as f:
            f.write(f" {int(ok)}")
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_targets_once():
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus(24, 10)
    for world in (1, 2, 3, 8):
        shards = shard_targets(g, world)
        allidx = np.sort(np.concatenate(shards))
        assert np.array_equal(allidx, np.arange(g.n_tgt))
        pairs = [g.group_source_counts()[g.ctr_group[g.tgt_center[s]]].sum() for s in shards]
        assert max(pairs) <= 1.25 * (sum(pairs) / world) + 2000


def test_gloo_world2_sharded_equals_full(scratch):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    res = scratch / "res.txt"
    mp.start_processes(_worker, args=(2, port, str(res)), nprocs=2, join=True, start_method="spawn")
    ok, c0, c1, ok_driver = map(int, res.read_text().split())
    assert ok == 1
    assert abs(c0 - c1) <= 0.1 * (c0 + c1)
    assert ok_driver == 1


def test_shard_geometry_keeps_sources_and_lists():
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus(24, 10)
    idx = shard_targets(g, 3)[1]
    sub = shard_geometry(g, idx)
    assert sub.tgt_xyz.shape == (3, len(idx)) and np.array_equal(sub.tgt_center, g.tgt_center[idx])
    assert sub.src_xyz is g.src_xyz and sub.range_begin is g.range_begin
    assert sub.tgt_normal is None or np.array_equal(sub.tgt_normal, g.tgt_normal[:, idx])


def _fake_world(geometry, evaluate_for, world):
    """distributed_eval for every rank of a world run in turn in this process:
    a first pass records what each rank contributes to each all-gather call,
    a second pass gives every rank's gather all the ranks' contributions."""
    sent = {r: [] for r in range(world)}

    def recorder(r):
        def all_gather(tensor_list, tensor):
            sent[r].append(tensor.clone())
            for t in tensor_list:
                t.zero_()
        return all_gather

    def replayer(r):
        calls = iter(range(len(sent[r])))

        def all_gather(tensor_list, tensor):
            i = next(calls)
            for q in range(world):
                tensor_list[q].copy_(tensor if q == r else sent[q][i])
        return all_gather

    for r in range(world):
        distributed_eval(geometry, evaluate_for(r), r, world, all_gather=recorder(r))
    return [distributed_eval(geometry, evaluate_for(r), r, world, all_gather=replayer(r)) for r in range(world)]


def test_distributed_eval_single_process_world3():
    """The driver with a fake all-gather over three ranks run in turn."""
    import oracle
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus(20, 8)
    ref = oracle.tsqbx_laplace(g, 5, mu, slp=True, dlp=True)
    got = _fake_world(g, lambda r: (lambda shard: oracle.tsqbx_laplace(shard, 5, mu, slp=True, dlp=True)), 3)
    for res in got:
        assert all(np.array_equal(res[k], ref[k]) for k in ("slp", "dlp"))


def test_distributed_eval_complex_and_torch_outputs():
    """Complex (Helmholtz) outputs travel as (re, im) pairs; torch outputs
    come back as torch tensors."""
    import torch
    import oracle
    from tsqbx_inputs import configs
    g, muh, _ = configs.torus_helmholtz(12, 5, k=3.0)
    ref = oracle.tsqbx_helmholtz(g, 4, 3.0, muh, slp=True, dlp=True)

    def evaluate_for(r):
        return lambda sh: {k: torch.from_numpy(v) for k, v in
                           oracle.tsqbx_helmholtz(sh, 4, 3.0, muh, slp=True, dlp=True).items()}

    for res in _fake_world(g, evaluate_for, 2):
        for k in ("slp", "dlp"):
            assert isinstance(res[k], torch.Tensor) and res[k].dtype == torch.complex128
            assert np.array_equal(res[k].numpy(), ref[k])


def test_more_ranks_than_targets():
    """Ranks beyond the target count get empty shards; the reassembled result
    is still the single-rank one."""
    import oracle
    from helpers import cloud_geometry
    g = cloud_geometry(np.random.default_rng(3), n_ctr=2, n_src=40, tgt_per_ctr=1)
    mu = np.random.default_rng(4).standard_normal(g.n_src)
    world = 5
    shards = shard_targets(g, world)
    assert sum(len(s) for s in shards) == g.n_tgt and sum(len(s) == 0 for s in shards) >= world - g.n_tgt
    ref = oracle.tsqbx_laplace(g, 4, mu, slp=True)["slp"]
    got = _fake_world(g, lambda r: (lambda sh: oracle.tsqbx_laplace(sh, 4, mu, slp=True)), world)
    for res in got:
        assert np.array_equal(res["slp"], ref)
