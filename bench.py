"""Benchmark of the near-field TSQBX step (Laplace p = 9, single + double layer)
on the torus workload: R = 1, r = 0.35, 256 x 96 quads (49,152 flat triangles,
294,912 sources), two QBX centers per node (589,824 targets), GIGAQBX octree
List 1 / 3 close / 4 close pair lists (n_max = 64, t_f = 0.9).

One step = one evaluation of both layers for one density vector.  The
headline `value` is the FP64 path; the same step in mixed precision is
reported beside it under "mixed".  Metric unit: pair-terms/s, a pair-term
being one order n <= p of one (target, source) pair.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank evaluates its own density on its own GPU
(independent matvecs, no data-path collective) and `value` is the pair-terms
of all ranks over the slowest rank's time (weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P = 9
METRIC = "TSQBX pair-terms/s at Laplace p=9 (single+double layer), FP64 vs mixed"
UNIT = "pair-terms/s"
WORKLOAD = "torus 256x96 quads, 294912 sources, 589824 targets, octree lists n_max=64, Laplace SLP+DLP p=9"

# Peaks (ALU-bound kernels): derived from unit counts and the maximum SM clock
# (152 SMs x FMA lanes/clock/SM x 2 flop x 2070 MHz); FP64 at 2 FMA/clk/SM
# (the GB300 nominal 1.25 TFLOP/s), FP32 at 128 FMA/clk/SM.
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
PEAK_FP64_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP32_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12


def flops_per_pair(p, precision):
    """Algorithmic flops per (target, source) pair of the SLP+DLP kernels
    (FMA = 2): geometry 19 (+6 for the float-float difference in mixed),
    10 per recurrence step n = 1..p-1, 32 for closing both layers, and 8 for
    the Kahan updates in mixed."""
    base = 19 + 10 * (p - 1) + 32
    return base + (6 + 8 if precision == "mixed" else 0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target duration of the bounded CPU oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload():
    from tsqbx_inputs import configs
    g, mu, tree = configs.torus()
    return g, mu


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        top = [s for s in sm if s >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(top), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- CPU side

def cpu_sample(g, mu, seconds, rng_seed=7):
    """Time the FP64 oracle (path A, Appendix A) on a bounded random sample of
    targets: calibrate on 1000 targets, then size the sample to `seconds`."""
    import oracle
    rng = np.random.default_rng(rng_seed)
    per_group = g.group_source_counts()
    tgt_pairs = per_group[g.ctr_group[g.tgt_center]]
    order = rng.permutation(g.n_tgt)
    cal = np.sort(order[:1000])
    t0 = time.perf_counter()
    oracle.tsqbx_laplace(g, P, mu, subset=cal, slp=True, dlp=True)
    rate = tgt_pairs[cal].sum() / max(time.perf_counter() - t0, 1e-6)
    want = int(rate * seconds)
    csum = np.cumsum(tgt_pairs[order])
    n = int(min(max(np.searchsorted(csum, want) + 1, 1000), g.n_tgt))
    idx = np.sort(order[:n])
    t0 = time.perf_counter()
    ref = oracle.tsqbx_laplace(g, P, mu, subset=idx, slp=True, dlp=True)
    dt = time.perf_counter() - t0
    pairs = int(tgt_pairs[idx].sum())
    return {"idx": idx, "ref": ref, "seconds": dt, "pairs": pairs,
            "value": pairs * (P + 1) / dt, "cores": oracle.num_threads()}


def reference_arm(args):
    """--impl reference: the FP64 CPU oracle on a bounded sample per step."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    g, mu = workload()
    per_group = g.group_source_counts()
    tgt_pairs = per_group[g.ctr_group[g.tgt_center]]
    rng = np.random.default_rng(11)
    n = 4000
    times, pairs_done = [], 0
    for step in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(g.n_tgt, n, replace=False))
        t0 = time.perf_counter()
        oracle.tsqbx_laplace(g, P, mu, subset=idx, slp=True, dlp=True)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            pairs_done += int(tgt_pairs[idx].sum())
    total = sum(times)
    value = pairs_done * (P + 1) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": f"{n} random targets"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{n} random targets per step of the torus workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU side

def time_device(plan, dmu, outs, stream, steps, warmup, flush, barrier):
    """W untimed warm-up steps, then K steps bracketed by barrier + synchronize.
    Per step: flush L2 (untimed), then CUDA events on `stream` around the
    evaluation; the library's own events give the expansion kernel alone."""
    import torch
    for _ in range(warmup):
        plan.eval_async(dmu, outs, stream=stream)
    barrier()
    torch.cuda.synchronize()
    step_ms, kern_ms = [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval_async(dmu, outs, stream=stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(plan.kernel_ms())
    torch.cuda.synchronize()
    barrier()
    return step_ms, kern_ms


def gpu_selector(dev, local_rank):
    """Identifier nvidia-smi -i accepts for this device (UUID when known)."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u and u != "None":
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return str(local_rank)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    import paper_1811_01110_gb300 as pkg

    g, mu = workload()
    if world > 1:    # each rank evaluates its own density (independent matvec)
        mu = mu * (1.0 + 0.01 * rank)
    plans = {prec: pkg.Plan(g, "laplace", ("slp", "dlp"), p=P, precision=prec, device=local_rank)
             for prec in ("fp64", "mixed")}
    info = plans["fp64"].info()
    pair_terms = info["n_pair_terms"]
    dmu = torch.from_numpy(mu).to(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    outs = {prec: {l: torch.empty(g.n_tgt, dtype=torch.float64, device=dev) for l in ("slp", "dlp")}
            for prec in plans}

    # ---- timed regions: K device-resident steps per precision
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    res = {}
    sampler = ClockSampler(gpu_selector(dev, local_rank))
    wall0 = time.perf_counter()
    with sampler:
        for prec in ("fp64", "mixed"):
            res[prec] = time_device(plans[prec], dmu, outs[prec], stream, args.steps, args.warmup,
                                    flush, barrier)
    wall_s = time.perf_counter() - wall0
    clocks = sampler.summary()

    def agg(ms_list):
        t = sum(ms_list) / 1e3
        if world > 1:
            tt = torch.tensor([t], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            t = float(tt.item())
        return t

    summary = {}
    for prec in ("fp64", "mixed"):
        step_ms, kern_ms = res[prec]
        t_step = agg(step_ms)
        t_kern = agg(kern_ms)
        value = pair_terms * args.steps * world / t_step
        kavg = t_kern / args.steps
        fl = flops_per_pair(P, prec) * info["n_pairs"]
        peak = PEAK_FP64_TFLOPS if prec == "fp64" else PEAK_FP32_TFLOPS
        achieved = fl / kavg / 1e12
        summary[prec] = {
            "value": value, "ms_per_step": 1e3 * t_step / args.steps,
            "kernel_ms": 1e3 * kavg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "pipe": "fp64" if prec == "fp64" else "fp32",
                         "peak_source": "derived: 152 SMs x %d FMA/clk x 2 flop x 2070 MHz"
                                        % (2 if prec == "fp64" else 128),
                         "flops_per_pair": flops_per_pair(P, prec)},
        }

    # ---- end to end through the public API with host buffers
    e2e = None
    host_mu = np.ascontiguousarray(mu)
    e2e_t = []
    for i in range(args.warmup + max(3, args.steps // 2)):
        t0 = time.perf_counter()
        host_out = plans["fp64"].eval(host_mu)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_t.append(dt)
    t_e2e = sum(e2e_t)
    if world > 1:
        tt = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(tt.item())
    e2e = {"value": pair_terms * len(e2e_t) * world / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(host_mu.nbytes),
           "d2h_bytes_per_step": int(2 * g.n_tgt * 8 + 4)}

    if rank != 0:
        return
    # ---- CPU baseline (oracle on a bounded sample) + error of both GPU paths there
    cpu = None
    err = {}
    if not args.no_cpu:
        cs = cpu_sample(g, mu, args.cpu_seconds)
        cpu = {"value": cs["value"], "unit": UNIT, "cores": cs["cores"], "kind": "oracle",
               "sample": f"{len(cs['idx'])} random targets ({cs['pairs']} pairs, "
                         f"{cs['seconds']:.1f} s) of the benchmark workload, SLP+DLP p=9"}
        for prec in ("fp64", "mixed"):
            for l in ("slp", "dlp"):
                got = outs[prec][l].cpu().numpy()[cs["idx"]]
                ref = cs["ref"][l]
                err[f"{prec}_{l}"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        for l in ("slp", "dlp"):
            ref = cs["ref"][l]
            err[f"e2e_fp64_{l}"] = float(np.max(np.abs(host_out[l][cs["idx"]] - ref)) / np.max(np.abs(ref)))

    f = summary["fp64"]
    line = {
        "metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "p": P, "layers": "slp+dlp", "n_pairs": info["n_pairs"],
                   "pair_terms_per_step": pair_terms, "n_items": info["n_items"],
                   "lane_utilisation": round(info["lane_utilisation"], 4),
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "timing": "CUDA events on the launching stream per step"},
        "roofline": f["roofline"],
        "kernel_ms": f["kernel_ms"],
        "mixed": {"value": summary["mixed"]["value"], "unit": UNIT, "dtype": "f32 recurrence, f64 sums",
                  "ms_per_step": summary["mixed"]["ms_per_step"], "kernel_ms": summary["mixed"]["kernel_ms"],
                  "roofline": summary["mixed"]["roofline"],
                  "speedup_vs_fp64": summary["mixed"]["value"] / f["value"]},
        "error_vs_oracle": err or None,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps * 2,
        "clocks": clocks,
        "wall_s_timed_region": wall_s,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    for p_ in plans.values():
        p_.close()


if __name__ == "__main__":
    main()
