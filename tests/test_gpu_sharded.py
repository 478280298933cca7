"""The sharded evaluation through the GPU library: two gloo ranks, both on
cuda:0 (the ranks' kernels never wait on one another: each rank evaluates its
own target shard with its own Plan, then the host-side gloo all-gather
reassembles the outputs), compared with the FP64 CPU oracle at the FP64
parity tolerance (1e-12 relative).  Targets are independent (Alg. 1 Stage 3),
so the shards need no exchange before the gather."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch
    import torch.distributed as dist
    import paper_1811_01110_gb300 as pkg
    from paper_1811_01110_gb300.sharding import distributed_eval
    from tsqbx_inputs import configs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    lines = []
    cases = [("laplace", configs.torus(32, 12)[:2], dict(p=9), ("slp", "dlp", "sp")),
             ("helmholtz", configs.torus_helmholtz(24, 10, k=5.0)[:2], dict(p=8, k=5.0), ("slp", "dlp", "sp"))]
    for kernel, (g, mu), kw, layers in cases:
        dmu = torch.from_numpy(np.ascontiguousarray(mu)).cuda()

        def evaluate(shard):
            with pkg.Plan(shard, kernel, layers, device=0, **kw) as plan:
                out = plan.eval(dmu)               # device outputs
                torch.cuda.synchronize()
                return out

        got = distributed_eval(g, evaluate, rank, world)
        if rank == 0:
            import oracle
            idx = np.sort(np.random.default_rng(7).choice(g.n_tgt, 600, replace=False))
            if kernel == "laplace":
                ref = oracle.tsqbx_laplace(g, kw["p"], mu, subset=idx, slp=True, dlp=True, sp=True)
            else:
                ref = oracle.tsqbx_helmholtz(g, kw["p"], kw["k"], mu, subset=idx, slp=True, dlp=True, sp=True)
            for layer in layers:
                v = got[layer].cpu().numpy()[idx]
                err = float(np.max(np.abs(v - ref[layer])) / np.max(np.abs(ref[layer])))
                lines.append(f"{kernel} {layer} {err:.3e} {int(got[layer].shape[0] == g.n_tgt)}")
    if rank == 0:
        with open(result_path, "w") as f:
            f.write("\n".join(lines))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu_match_the_oracle(scratch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    res = scratch / "res.txt"
    mp.start_processes(_worker, args=(2, _free_port(), str(res)), nprocs=2, join=True, start_method="spawn")
    rows = [l.split() for l in res.read_text().splitlines()]
    assert len(rows) == 6
    for kernel, layer, err, full in rows:
        assert float(err) <= TOL, (kernel, layer, err)
        assert full == "1"
