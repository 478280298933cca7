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

# Fallback peaks of the ALU-bound kernels, used only when the register-only
# probe (tsqbx_measure_pipe_peaks) cannot run: the device's SM count x FMA
# lanes per clock per SM (FP64 2, FP32 128) x 2 flop x the maximum SM clock.
SM_MAX_MHZ = 2070.0
HEADLINE_MAX_BYTES = 2000       # the last stdout line stays well inside a 3-4 KB tail


def derived_peaks(sm_count):
    return {"fp64": sm_count * 2 * 2 * SM_MAX_MHZ * 1e6 / 1e12,
            "fp32": sm_count * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12,
            "source": f"derived: {sm_count} SMs x (2 | 128) FMA/clk x 2 flop x {SM_MAX_MHZ:.0f} MHz"}


def a_priori_flops_per_pair(p, dlp=True):
    """The a priori count of the Laplace kernel's work per pair (FMA = 2):
    6p + 20 for the single layer (geometry about 20, about 6 per order), plus
    4 per pair-term (p + 1 of them) and 20 per pair for the double layer.
    134 at p = 9 with both layers."""
    return 6 * p + 20 + ((4 * (p + 1) + 20) if dlp else 0)


# FP32 flops (FMA = 2) of the double-float building blocks (csrc/dfloat.cuh):
# TwoSum 6, FastTwoSum 3, TwoProd 3; DWPlusDW 11, DWTimesDW 10, DWTimesFP 8;
# a 3-vector dot product 52; 1/sqrt with two Newton steps 81.
_DF_ADD, _DF_MUL, _DF_MULF, _DF_DOT, _DF_RSQRT = 11, 10, 8, 52, 81


def _lambda_is_float(n):
    """Whether the Q' coefficient lambda_n = prod_{m<n} (2m+1)/m is exactly a
    float (a dyadic rational with a short enough numerator: n <= 12)."""
    lam = 1.0
    for m in range(1, n):
        lam *= (2.0 * m + 1.0) / m
    return float(np.float32(lam)) == lam


def df64_fp32_flops_per_pair(p, dlp=True, sp=False):
    """FP32 flops per pair (FMA = 2) of the double-float Laplace kernel
    (laplace_df_items.cuh, multi-target items): geometry (s - c as three
    double-float differences, R^2, 1/R, 1/R^2, qx, q2, w/R) 258; the Clenshaw
    single layer 21 + 52 per order step + 21; with the double layer or S'
    the Q' recurrence 62 per step n = 2..p-1 (the n = 1 step is exact; 60
    where lambda_n is a float, n <= 12, and its product takes DWTimesFP), its
    top 61 (57 when lambda_p and lambda_{p+1} are floats), the closing sums
    83, the single layer's accumulation 21 and w/R^3 10; the double layer 167
    (two dots, the combination, accumulation), S' 104.  1016 at p = 9 with
    both layers."""
    geo = 3 * _DF_ADD + _DF_DOT + _DF_RSQRT + _DF_MUL + (_DF_DOT + _DF_MUL) + 2 * _DF_MUL
    q = max(p - 1, 0)
    if not dlp and not sp:
        return geo + (_DF_ADD + _DF_MUL) + (3 * _DF_MUL + 2 * _DF_ADD) * q + (_DF_ADD + _DF_MUL)

    def lam_mul(n):     # lambda_n times a double-float: DWTimesFP when lambda_n is a float
        return _DF_MULF if _lambda_is_float(n) else _DF_MUL
    f = geo + sum(2 * _DF_ADD + 3 * _DF_MUL + lam_mul(n) for n in range(2, p))
    if p >= 1:
        f += 3 * _DF_MUL + lam_mul(p) + lam_mul(p + 1) + _DF_ADD            # Q'_p, Q'_{p+1}
    f += _DF_ADD + (_DF_MULF + 2 * _DF_ADD) + (2 * _DF_MUL + 2 * _DF_ADD)     # S2, c1, S
    f += _DF_MUL + _DF_ADD + _DF_MUL                                          # acc_s, w/R^3
    if dlp:
        f += 2 * _DF_DOT + 3 * _DF_MUL + 3 * _DF_ADD
    if sp:
        f += _DF_DOT + 3 * _DF_MUL + 2 * _DF_ADD
    return f


def flops_per_pair(p, precision, dlp=True, sp=False):
    """Algorithmic flops per (target, source) pair (FMA = 2) of the Laplace
    kernels.  Single layer alone: geometry 19 (d, R^2, 1/R, qx, q2), 2 for
    b_{p-1}, 5 per Clenshaw step k = p-2..0, closing 3.  With the double layer or S' (one
    recurrence for Q'_n): geometry 20; the recurrence from n = 2 (its n = 1
    step, U_2 = qx and the first closing sum, is exact), 5 at n = 2 (U_1 = 1)
    and 6 per step n = 3..p-1; the top step
    and sums 7, sum Q_n from the closing identity 7, accumulation 2; the
    double layer adds 17 (two normal dots, (b - a) S2 - a Q'_{p+1} and its
    accumulation), S' 10 (one dot, the combination, accumulation; +1 for
    1/R^3 without the double layer).  Mixed precision adds 6 for the
    float-float difference and 1 per layer for the sum (plain within a
    shared-memory tile; the Kahan update once per tile is not counted)."""
    if not dlp and not sp:
        f = 19 + (2 + 5 * (p - 1) if p >= 1 else 0) + 3
    else:
        f = 20 + (5 + 6 * (p - 3) if p >= 3 else 0) + 16
        if dlp:
            f += 17
        if sp:
            f += 10 + (0 if dlp else 1)
    if precision == "mixed":
        f += 6 + (1 + int(dlp) + int(sp))
    return f


def helmholtz_flops_per_pair(p, dlp=False, sp=False):
    """Helmholtz kernel (FP64), flops per pair (FMA = 2).  Every layer is a
    Clenshaw sum over the Hankel factors in real arithmetic.
    * Common to all: geometry and 1/z 20, sincos counted as 2, the Legendre
      recurrence forward 3 per order step, (2n+1)/z 1 per order, and for the
      single layer the combination with g_0, g_1 5 plus the closing with
      e^{iz} and the complex weight 16.
    * Single layer alone: 4 per order backward (the product folded into an
      FMA).  That is 8 p + 40 in all.
    * With the double layer: T'_n forward 4 per step, and 14 per order
      backward for both sums (a_n, the single layer's step, e_n, the double
      layer's coefficient and step).  Closing: normal dots 17, combination 11,
      e^{iz} and weight 16.
    * S': T'_n forward 4 per step (unless the double layer has it), 7 per
      order backward, normal dot 10, combination 5, e^{iz} and weight 16.
    * The backward step n = p starts from b_{p+1} = b_{p+2} = 0 and is taken
      as b_p = c_p: it saves (2p+1)/z and the step's products by zero, 4
      flops with the single layer alone, 8 with the double layer, 3 more
      with S'."""
    q = max(p - 1, 0)
    f = 20 + 2 + 3 * q + p + 5 + 16
    f += 14 * p + 4 * q + 17 + 11 + 16 if dlp else 4 * p
    if sp:
        f += 7 * p + (0 if dlp else 4 * q) + 10 + 5 + 16
    if p >= 1:
        f -= (8 if dlp else 4) + (3 if sp else 0)
    return f


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the bounded CPU oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline workload (no batched / Helmholtz / sphere legs)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the automatic schedules")
    ap.add_argument("--detail", default=os.path.join(ROOT, "bench_detail.json"),
                    help="file for the full result (every workload); stdout gets the headline line only")
    ap.add_argument("--only", choices=["batched", "helmholtz", "sphere", "serving", "target_derivative",
                                       "conventional", "lists", "multi_density"],
                    help="run one secondary workload alone and print its JSON (for profiling)")
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
    oracle.tsqbx_laplace(g, P, mu, subset=cal[:64], slp=True, dlp=True)   # start the thread pool
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
    cores = oracle.num_threads()
    # the same oracle on one core, over a fifth of the time budget
    n1 = max(50, int(len(idx) / max(cores, 1) / 5))
    idx1 = np.sort(order[:n1])
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.tsqbx_laplace(g, P, mu, subset=idx1, slp=True, dlp=True)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    return {"idx": idx, "ref": ref, "seconds": dt, "pairs": pairs,
            "value": pairs * (P + 1) / dt, "cores": cores,
            "single_core": {"value": int(tgt_pairs[idx1].sum()) * (P + 1) / dt1, "targets": int(n1),
                            "seconds": dt1}}


def oracle_sample(g, run, seconds, terms_per_pair, seed=7, cal=200):
    """Time the FP64 oracle, `run(subset) -> {layer: values}`, on a random
    sample of targets sized to about `seconds` after a calibration run on
    `cal` targets.  Returns the sample, its reference values and the rate."""
    import oracle
    rng = np.random.default_rng(seed)
    tgt_pairs = g.group_source_counts()[g.ctr_group[g.tgt_center]]
    order = rng.permutation(g.n_tgt)
    n0 = min(cal, g.n_tgt)
    c = np.sort(order[:n0])
    run(c[:16])                                     # start the thread pool
    t0 = time.perf_counter()
    run(c)
    rate = tgt_pairs[c].sum() / max(time.perf_counter() - t0, 1e-6)
    csum = np.cumsum(tgt_pairs[order])
    n = int(min(max(np.searchsorted(csum, rate * seconds) + 1, n0), g.n_tgt))
    idx = np.sort(order[:n])
    t0 = time.perf_counter()
    ref = run(idx)
    dt = time.perf_counter() - t0
    pairs = int(tgt_pairs[idx].sum())
    return {"idx": idx, "ref": ref, "seconds": dt, "pairs": pairs,
            "value": pairs * terms_per_pair / dt, "cores": oracle.num_threads()}


def host_cpu():
    """The host's CPU model (lscpu 'Model name') and logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def max_rel_err(got, ref):
    """max_t |got - ref| / max_t |ref| over one output array."""
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


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
                         **host_cpu(), "sample": f"{n} random targets per step of the torus workload"},
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


# DRAM bytes (read + write) per launch of each timed kernel, from one ncu
# capture of the current kernel versions (summaries in profiles/: the
# laplace_*_p9_torus256x96.md files, helmholtz_slp_p12_torus444x166.md and
# batch_laplace_mixed_ellipsoids64.md).  The torus kernels were captured at
# the default staging depth (64); the timed plans are autotuned.
# A kernel changed since its capture must map to None here.
TRAFFIC_BYTES = {
    ("laplace", "fp64", "slp+dlp"): 87.96e6,
    ("laplace", "mixed", "slp+dlp"): 55.96e6,
    ("laplace", "df64", "slp+dlp"): 74.24e6,
    ("helmholtz", "fp64", "slp"): 321.79e6,
    ("batched", "mixed", "slp"): 299.55e6,
}


def measured_hbm_gbs():
    """The machine's measured copy bandwidth (MEASURED_PEAKS.json), else the
    fallback figure of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


PEAKS = None     # set once per run by measure_peaks()


def measure_peaks(pkg, dev_index, sm_count):
    """FP64 and FP32 pipe peaks for the rooflines: the library's register-only
    FMA probe on this device (the packed-FP32 figure when it is higher, since
    the mixed kernel issues packed instructions), else the derived figures."""
    global PEAKS
    try:
        m = pkg.measure_pipe_peaks(dev_index)
        PEAKS = {"fp64": m["fp64_tflops"], "fp32": max(m["fp32_tflops"], m["fp32x2_tflops"]),
                 "source": "measured: register-only FMA probe (tsqbx_measure_pipe_peaks), %d SMs, best of 3 "
                           "launches of ~150 ms" % m["sm_count"], "probe": m}
    except Exception as exc:             # the kernels' numbers stand against the derived peaks
        PEAKS = dict(derived_peaks(sm_count), probe_error=repr(exc)[:200])
    PEAKS["derived"] = derived_peaks(sm_count)
    return PEAKS


def roofline(flops_per_launch, kernel_s, pipe, traffic_key=None):
    """ALU roofline of one launch: algorithmic flops over the kernel's CUDA-event
    time, against the FP64 or FP32 pipe peak (measured when the probe ran)."""
    peaks = PEAKS or derived_peaks(152)
    peak = peaks[pipe]
    achieved = flops_per_launch / kernel_s / 1e12
    traffic = TRAFFIC_BYTES.get(traffic_key)
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic,
           "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
           "pipe": pipe, "peak_source": peaks["source"]}
    if traffic is not None:
        # the DRAM side of the same launch: ncu bytes over this run's kernel time
        hbm, src = measured_hbm_gbs()
        out["hbm"] = {"achieved_gbs": traffic / kernel_s / 1e9, "peak_gbs": hbm,
                      "frac": traffic / kernel_s / 1e9 / hbm, "peak_source": src}
    return out


def leg_batched(pkg, torch, dev, steps, warmup, flush, check_targets=0):
    """64 ellipsoids (1k-200k sources, Laplace SLP, p in {5,7,9}, mixed) in one
    persistent launch replayed from a CUDA graph, against the same 64 plans
    evaluated one after another.  With check_targets > 0 the batched results
    of every eighth surface are compared with the FP64 oracle on that many
    seeded random targets each."""
    from tsqbx_inputs import configs
    surfaces = configs.ellipsoid_batch()
    plans = [pkg.Plan(g, "laplace", ("slp",), p=g.meta["p"], precision="mixed", device=dev.index)
             for g, _ in surfaces]
    dens = [torch.from_numpy(mu).to(dev) for _, mu in surfaces]
    outs = [{"slp": torch.empty(g.n_tgt, dtype=torch.float64, device=dev)} for g, _ in surfaces]
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    res = {}
    with pkg.Batch(plans, use_graph=True) as batch:
        info = batch.info()
        for _ in range(warmup):
            batch.eval_async(dens, outs, stream=stream)
        torch.cuda.synchronize()
        ms, kms = [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch.eval_async(dens, outs, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            kms.append(batch.kernel_ms())
        torch.cuda.synchronize()
    checked = list(range(0, len(surfaces), 8)) if check_targets > 0 else []
    batch_vals = {i: outs[i]["slp"].cpu().numpy().copy() for i in checked}
    # the same work as 64 separate evaluations on one stream
    seq = []
    for i in range(warmup + steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pl, d, o in zip(plans, dens, outs):
            pl.eval_async(d, o, stream=stream)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            seq.append(e0.elapsed_time(e1))
    pt = info["n_pair_terms"]
    t = sum(ms) / 1e3 / steps
    fl = sum(flops_per_pair(pl.p, "mixed", dlp=False) * pl.info()["n_pairs"] for pl in plans)
    res = {"workload": "64 seeded ellipsoids (semi-axes U(0.5,2)), %d sources, %d pairs, Laplace SLP, "
                       "p in {5,7,9}, lists of 50-800 sources per center" % (
                           sum(g.n_src for g, _ in surfaces), info["n_pairs"]),
           "value": pt / t, "unit": UNIT, "dtype": "f32 recurrence, f64 sums", "ms_per_step": 1e3 * t,
           "kernel_ms": sum(kms) / steps, "launches_per_step": info["launches_per_eval"],
           "persistent_ctas": info["grid_blocks"], "graph": bool(info["graph"]),
           "sequential_ms_per_step": sum(seq) / steps,
           "speedup_vs_sequential": (sum(seq) / steps) / (1e3 * t),
           "roofline": roofline(fl, sum(kms) / steps / 1e3, "fp32", ("batched", "mixed", "slp"))}
    if checked:
        try:
            import oracle
            worst = 0.0
            rng = np.random.default_rng(17)
            for i in checked:
                g, mu = surfaces[i]
                idx = np.sort(rng.choice(g.n_tgt, min(check_targets, g.n_tgt), replace=False))
                ref = oracle.tsqbx_laplace(g, g.meta["p"], mu, subset=idx, slp=True)["slp"]
                worst = max(worst, max_rel_err(batch_vals[i][idx], ref))
            res["error_vs_oracle"] = {"slp": worst, "surfaces": len(checked), "targets_each": int(check_targets)}
        except Exception as exc:      # the GPU numbers stand without the check
            res["error_vs_oracle"] = {"unavailable": repr(exc)[:200]}
    for pl in plans:
        pl.close()
    return res


def leg_helmholtz(pkg, torch, dev, steps, warmup, flush, cpu_seconds=0.0):
    """Torus 444 x 166 quads (884,448 sources, 1,768,896 targets), octree
    lists, Helmholtz k = 10, p = 12, FP64, plane-wave density: the single
    layer alone, single + double layer (the combined-field operator's
    parts, one pass), and all three layers with S'.  With cpu_seconds > 0
    the FP64 oracle is timed on a random target sample of the single layer
    (about that long), and every layer's GPU result is compared with it."""
    from tsqbx_inputs import configs
    g, mu, _ = configs.torus_helmholtz()
    dmu = torch.from_numpy(mu).to(dev)
    stream = torch.cuda.Stream(device=dev)
    res = {"workload": "torus 444x166 quads, 884448 sources, 1768896 targets, octree lists, "
                       "Helmholtz k=10 p=12", "unit": UNIT, "dtype": "f64"}
    for name, layers in (("slp", ("slp",)), ("slp+dlp", ("slp", "dlp")), ("slp+dlp+sp", ("slp", "dlp", "sp"))):
        plan = pkg.Plan(g, "helmholtz", layers, p=12, k=10.0, device=dev.index)
        info = plan.info()
        out = {l: torch.empty(g.n_tgt, dtype=torch.complex128, device=dev) for l in layers}
        step_ms, kern_ms = time_device(plan, dmu, out, stream, steps, warmup, flush, lambda: None)
        t = sum(kern_ms) / 1e3 / steps
        fl = helmholtz_flops_per_pair(12, "dlp" in layers, "sp" in layers)
        res["n_pairs"] = info["n_pairs"]
        res[name] = {"value": info["n_pair_terms"] / (sum(step_ms) / 1e3 / steps),
                     "ms_per_step": sum(step_ms) / steps, "kernel_ms": 1e3 * t,
                     "roofline": dict(roofline(fl * info["n_pairs"], t, "fp64", ("helmholtz", "fp64", name)),
                                      flops_per_pair=fl)}
        if cpu_seconds > 0:
            res[name]["error_vs_oracle"] = _helmholtz_oracle_check(res, g, mu, layers, out, cpu_seconds)
        plan.close()
    res["value"] = res["slp"]["value"]
    return res


def _helmholtz_oracle_check(res, g, mu, layers, out, cpu_seconds):
    """The oracle on target samples of the Helmholtz workload: the timed
    single-layer sample (which also gives the CPU baseline), and for the plans
    with more layers 200 targets of it, all their layers."""
    import oracle
    try:
        if layers == ("slp",):
            cs = oracle_sample(g, lambda s: oracle.tsqbx_helmholtz(g, 12, 10.0, mu, subset=s, slp=True),
                               cpu_seconds, 13)
            res["_sample"] = cs["idx"]
            res["cpu_baseline"] = {"value": cs["value"], "unit": UNIT, "cores": cs["cores"], "kind": "oracle",
                                   "sample": f"{len(cs['idx'])} random targets ({cs['pairs']} pairs, "
                                             f"{cs['seconds']:.1f} s), single layer"}
            return {"slp": max_rel_err(out["slp"].cpu().numpy()[cs["idx"]], cs["ref"]["slp"]),
                    "targets": int(len(cs["idx"]))}
        sub = res["_sample"][:200]
        ref = oracle.tsqbx_helmholtz(g, 12, 10.0, mu, subset=sub, slp=True, dlp="dlp" in layers,
                                     sp="sp" in layers)
        e = {l: max_rel_err(out[l].cpu().numpy()[sub], ref[l]) for l in layers}
        e["targets"] = int(len(sub))
        return e
    except Exception as exc:          # the GPU numbers stand without the check
        return {"unavailable": repr(exc)[:200]}


def leg_conventional(pkg, torch, dev, steps, warmup, flush, check_targets=0):
    """Torus 96 x 36 quads (41,472 sources, 82,944 centers, octree lists) with
    1, 4, 16 and 64 targets per center, and with a mix (each center 1..64,
    log-uniform), SLP+DLP FP64, Laplace at p = 9 and Helmholtz (k = 10,
    plane-wave density) at p = 12: the target-specific path alone ("off"),
    conventional QBX for every center ("all"), and the cost model's
    per-center choice ("auto").  With check_targets > 0 every mode's result is
    compared with the FP64 oracle on that many seeded random targets."""
    from tsqbx_inputs import configs
    stream = torch.cuda.Stream(device=dev)
    base = "torus 96x36 quads, 41472 sources, 82944 centers, octree lists, targets per center in {1,4,16,64} " \
           "or mixed 1..64 log-uniform (uniform in each center's half-radius ball), SLP+DLP FP64, "
    res = {"workload": base + "Laplace p=9", "unit": UNIT, "cases": []}
    hel = {"workload": base + "Helmholtz k=10 p=12", "unit": UNIT, "cases": []}
    for tpc in (1, 4, 16, 64, "mixed:64"):
        g, mu, _ = configs.torus_near_targets(96, 36, tpc)
        for kernel, p, dest in (("laplace", 9, res), ("helmholtz", 12, hel)):
            if kernel == "helmholtz":
                hmu = np.ascontiguousarray(mu * np.exp(1j * 10.0 * g.src_xyz[0]))
                dmu = torch.from_numpy(hmu).to(dev)
                dt, kw = torch.complex128, {"k": 10.0}
            else:
                dmu = torch.from_numpy(mu).to(dev)
                dt, kw = torch.float64, {}
            case = {"targets_per_center": tpc, "n_targets": g.n_tgt}
            ref = idx = None
            if check_targets > 0:
                try:
                    import oracle
                    idx = np.sort(np.random.default_rng(19).choice(g.n_tgt, min(check_targets, g.n_tgt),
                                                                   replace=False))
                    ref = (oracle.tsqbx_helmholtz(g, p, 10.0, hmu, subset=idx, slp=True, dlp=True)
                           if kernel == "helmholtz" else
                           oracle.tsqbx_laplace(g, p, mu, subset=idx, slp=True, dlp=True))
                except Exception as exc:      # the GPU numbers stand without the check
                    case["error_vs_oracle"] = {"unavailable": repr(exc)[:200]}
            for mode in ("off", "all", "auto"):
                plan = pkg.Plan(g, kernel, ("slp", "dlp"), p=p, conventional=mode, device=dev.index, **kw)
                info = plan.info()
                outs = {l: torch.empty(g.n_tgt, dtype=dt, device=dev) for l in ("slp", "dlp")}
                step_ms, kern_ms = time_device(plan, dmu, outs, stream, steps, warmup, flush, lambda: None)
                t = sum(step_ms) / 1e3 / steps
                case[mode] = {"ms_per_step": 1e3 * t, "pair_terms_per_s": info["n_pair_terms"] / t,
                              "conv_centers": info["n_conv_centers"], "conv_targets": info["n_conv_targets"]}
                if ref is not None:
                    case[mode]["error_vs_oracle"] = {l: max_rel_err(outs[l].cpu().numpy()[idx], ref[l])
                                                     for l in ("slp", "dlp")}
                case["n_pairs"] = info["n_pairs"]
                plan.close()
            case["auto_vs_best"] = case["auto"]["ms_per_step"] / min(case["off"]["ms_per_step"],
                                                                       case["all"]["ms_per_step"])
            dest["cases"].append(case)
            del dmu
    res["helmholtz"] = hel
    return res


def leg_lists(pkg, torch, dev, steps, warmup, flush):
    """Octree + near-field lists (List 1 + List 3 close + List 4 close) on the
    GPU against the host builder of the input tooling (single-threaded C++),
    on the benchmark torus, the Helmholtz torus and the urchin gamma_8 (6
    icosphere subdivisions); n_max = 64, t_f = 0.9, n_mpole = 40.  The GPU
    time is the wall time of tsqbx_octree_build, host copies in and out
    included; every array is checked equal to the host builder's."""
    from tsqbx_inputs import configs, lists as L
    res = {"unit": "ms", "cases": []}
    for name, fn in (("torus 256x96", lambda: configs.torus_points(256, 96)),
                     ("torus 444x166", lambda: configs.torus_points(444, 166)),
                     ("urchin k=8, 6 subdivisions", lambda: configs.urchin_points(8, 6))):
        src, ctr, rad = fn()
        gpu_ms = []
        for i in range(warmup + steps):
            t = pkg.Octree(src, ctr, rad, device=dev.index)
            if i >= warmup:
                gpu_ms.append(t.stats["build_ms"])
        t0 = time.perf_counter()
        ref = L.Octree(src, ctr, rad)
        host_ms = 1e3 * (time.perf_counter() - t0)
        same = all(np.array_equal(np.asarray(getattr(t, a)), np.asarray(getattr(ref, a)))
                   for a in ("level", "parent", "src_perm", "ctr_box", "near_start", "near_begin", "near_end",
                             "src_begin", "src_end"))
        res["cases"].append({"workload": name, "n_sources": len(src), "n_centers": len(ctr),
                             "n_boxes": t.n_boxes, "max_level": t.stats["max_level"],
                             "near_ranges": t.stats["near_nnz"],
                             "center_source_pairs": t.stats["center_source_pairs"],
                             "gpu_ms": statistics.median(gpu_ms), "host_ms": host_ms,
                             "speedup": host_ms / statistics.median(gpu_ms), "identical_to_host": bool(same),
                             "gpu_phases_ms": {k: round(t.stats[k], 2) for k in
                                               ("upload_ms", "tree_ms", "order_ms", "lists_ms", "download_ms")}})
    return res


def leg_target_derivative(pkg, torch, dev, g, mu, steps, warmup, flush, check_targets=0):
    """The benchmark torus with S' added: Laplace single + double layer + S'
    (target-normal derivative) in one pass, p = 9, in every precision.  With
    check_targets > 0, every layer of every precision is compared with the
    FP64 oracle on that many seeded random targets."""
    dmu = torch.from_numpy(mu).to(dev)
    stream = torch.cuda.Stream(device=dev)
    layers = ("slp", "dlp", "sp")
    res = {"workload": WORKLOAD.replace("SLP+DLP", "SLP+DLP+S'"), "unit": UNIT}
    ref = idx = None
    if check_targets > 0:
        try:
            import oracle
            idx = np.sort(np.random.default_rng(13).choice(g.n_tgt, min(check_targets, g.n_tgt), replace=False))
            ref = oracle.tsqbx_laplace(g, P, mu, subset=idx, slp=True, dlp=True, sp=True)
        except Exception as exc:      # the GPU numbers stand without the check
            res["error_vs_oracle"] = {"unavailable": repr(exc)[:200]}
    for prec in ("fp64", "mixed", "df64"):
        plan = pkg.Plan(g, "laplace", layers, p=P, precision=prec, device=dev.index)
        info = plan.info()
        out = {l: torch.empty(g.n_tgt, dtype=torch.float64, device=dev) for l in layers}
        step_ms, kern_ms = time_device(plan, dmu, out, stream, steps, warmup, flush, lambda: None)
        t = sum(kern_ms) / 1e3 / steps
        fl = (df64_fp32_flops_per_pair(P, dlp=True, sp=True) if prec == "df64"
              else flops_per_pair(P, prec, dlp=True, sp=True))
        res[prec] = {"value": info["n_pair_terms"] / (sum(step_ms) / 1e3 / steps),
                     "ms_per_step": sum(step_ms) / steps, "kernel_ms": 1e3 * t,
                     "roofline": dict(roofline(fl * info["n_pairs"], t, "fp64" if prec == "fp64" else "fp32"),
                                      flops_per_pair=fl)}
        if ref is not None:
            res[prec]["error_vs_oracle"] = {l: max_rel_err(out[l].cpu().numpy()[idx], ref[l]) for l in layers}
            res[prec]["error_vs_oracle"]["targets"] = int(len(idx))
        plan.close()
    return res


def leg_multi_density(pkg, torch, dev, g, steps, warmup, flush):
    """The benchmark torus, Laplace single layer and single + double layer,
    p = 9, FP64 and df64: one density per evaluation against four in one
    (tsqbx_submit_multi_layers, device buffers), each timed on the host
    around submit and poll with the L2 flushed before every step (both the
    same way, on one plan).  Throughput counts the pair-terms of every
    density; the four results are checked bit for bit against the
    single-density evaluations."""
    rng = np.random.default_rng(2718)
    dens = [torch.from_numpy(rng.standard_normal(g.n_src)).to(dev) for _ in range(4)]
    res = {"workload": WORKLOAD.replace(", Laplace SLP+DLP p=9", "") + ", 4 densities per evaluation",
           "unit": UNIT}
    for layers in (("slp",), ("slp", "dlp")):
        key = "+".join(layers)
        res[key] = {}
        for prec in ("fp64", "df64"):
            plan = pkg.Plan(g, "laplace", layers, p=P, precision=prec, device=dev.index, max_rhs=4)
            pt = plan.info()["n_pair_terms"]
            outs = [{l: torch.empty(g.n_tgt, dtype=torch.float64, device=dev) for l in layers} for _ in range(4)]
            row = {}
            for n in (1, 4):
                dt = []
                for i in range(warmup + steps):
                    flush.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    t, _ = plan.submit_multi(dens[:n], outs=outs[:n])
                    pkg.poll(t, -1)
                    if i >= warmup:
                        dt.append(time.perf_counter() - t0)
                row[f"ms_{n}"] = 1e3 * sum(dt) / len(dt)
                row[f"value_{n}"] = n * pt * len(dt) / sum(dt)
            same = True
            for r in range(4):
                t, alone = plan.submit_multi(dens[r:r + 1])
                pkg.poll(t, -1)
                same = same and all(bool(torch.equal(alone[0][l], outs[r][l])) for l in layers)
            row["time_ratio_4_vs_1"] = row["ms_4"] / row["ms_1"]
            row["bit_identical"] = same
            res[key][prec] = row
            plan.close()
    return res


def leg_sphere(pkg, torch, dev, steps, warmup, flush, cpu_seconds=0.0):
    """Icosphere (3 subdivisions, 7,680 sources), radius-4h lists, Laplace SLP
    p = 5, FP64.  With cpu_seconds > 0 the FP64 oracle is timed on (up to)
    the whole workload and the GPU result compared with it."""
    from tsqbx_inputs import configs
    g, mu = configs.sphere()
    plan = pkg.Plan(g, "laplace", ("slp",), p=5, device=dev.index)
    info = plan.info()
    dmu = torch.from_numpy(mu).to(dev)
    out = {"slp": torch.empty(g.n_tgt, dtype=torch.float64, device=dev)}
    stream = torch.cuda.Stream(device=dev)
    step_ms, kern_ms = time_device(plan, dmu, out, stream, steps, warmup, flush, lambda: None)
    t = sum(kern_ms) / 1e3 / steps
    res = {"workload": "icosphere 1280 triangles, 7680 sources, radius-4h lists, Laplace SLP p=5",
           "n_pairs": info["n_pairs"], "value": info["n_pair_terms"] / (sum(step_ms) / 1e3 / steps),
           "unit": UNIT, "dtype": "f64", "ms_per_step": sum(step_ms) / steps, "kernel_ms": 1e3 * t,
           "roofline": roofline(flops_per_pair(5, "fp64", dlp=False) * info["n_pairs"], t, "fp64")}
    if cpu_seconds > 0:
        import oracle
        try:
            cs = oracle_sample(g, lambda s: oracle.tsqbx_laplace(g, 5, mu, subset=s, slp=True), cpu_seconds, 6)
            res["cpu_baseline"] = {"value": cs["value"], "unit": UNIT, "cores": cs["cores"], "kind": "oracle",
                                   "sample": f"{len(cs['idx'])} of {g.n_tgt} targets ({cs['pairs']} pairs, "
                                             f"{cs['seconds']:.2f} s)"}
            res["error_vs_oracle"] = {"slp": max_rel_err(out["slp"].cpu().numpy()[cs["idx"]], cs["ref"]["slp"]),
                                      "targets": int(len(cs["idx"]))}
        except Exception as exc:      # the GPU numbers stand without the check
            res["error_vs_oracle"] = {"unavailable": repr(exc)[:200]}
    plan.close()
    return res


def leg_serving(pkg, duration_s=10.0, rate=200.0, seed=20191114, size_priority=False, laplace_fp64_path="df64"):
    """Serving: Poisson arrivals over 16 resident geometries (5k-300k sources);
    each request a Laplace FP64, Laplace mixed or Helmholtz (k in {1,5,10})
    single-layer evaluation with p in {5,9,12} and a new seeded density.
    Plans are built first (warm start); each phase offers `duration_s` of
    arrivals; if the offered rate exceeds capacity a second phase runs at
    80 % of the measured capacity.  size_priority:
    the server's size-priority policy (short requests overtake long ones).
    laplace_fp64_path: the kernels that serve Laplace FP64 requests ("df64":
    the double-float kernels, which meet the FP64 bar of 1e-12)."""
    import threading
    from tsqbx_inputs import configs
    geoms = configs.serving_geometries()
    kinds = [("laplace", "fp64", 0.0), ("laplace", "mixed", 0.0), ("helmholtz", "fp64", 1.0),
             ("helmholtz", "fp64", 5.0), ("helmholtz", "fp64", 10.0)]
    srv = pkg.Server(hbm_budget=96 << 30, max_inflight=64, size_priority=size_priority,
                     laplace_fp64_path=laplace_fp64_path)
    gids = [srv.add_geometry(g, with_normals=False) for g in geoms]
    for gid in gids:
        for kernel, prec, k in (("laplace", "fp64", 0.0), ("laplace", "mixed", 0.0), ("helmholtz", "fp64", 1.0)):
            srv.prepare(gid, kernel, ("slp",), 5, k, prec)
    rng = np.random.default_rng(seed)
    dens_pool = [rng.standard_normal(g.n_src) for g in geoms]

    def phase(rate_hz, seconds):
        srv.reset_stats()
        n = int(rate_hz * seconds)
        gaps = rng.exponential(1.0 / rate_hz, n)
        reqs = []
        peak_queued = peak_running = 0
        t0 = time.perf_counter()
        due = t0
        for i in range(n):
            due += gaps[i]
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            gi = int(rng.integers(len(geoms)))
            kernel, prec, k = kinds[int(rng.integers(len(kinds)))]
            p = int(rng.choice([5, 9, 12]))
            mu = dens_pool[gi] * (1.0 + 0.01 * i)
            if kernel == "helmholtz":
                mu = mu * np.exp(1j * 0.1 * i)
            rid, _ = srv.submit(gids[gi], mu, kernel, ("slp",), p, k, prec)
            reqs.append(rid)
            if i % 25 == 0:                       # queue depth seen by arrivals
                live = srv.stats()
                peak_queued = max(peak_queued, live["queued"])
                peak_running = max(peak_running, live["running"])
        t_submit = time.perf_counter() - t0
        for rid in reqs:
            srv.poll(rid, timeout_us=-1)
        st = srv.stats()
        return {"offered_req_per_s": rate_hz, "requests": n, "submit_s": t_submit,
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                "completed": st["completed"], "failed": st["failed"], "rejected": st["rejected"],
                "merged": st["merged"],
                "peak_queued": int(peak_queued), "peak_running": int(peak_running),
                "achieved_req_per_s": st["completed"] / max(st["span_s"], 1e-9),
                "pair_terms_per_s": st["pair_terms_completed"] / max(st["span_s"], 1e-9),
                "span_s": st["span_s"]}

    first = phase(rate, duration_s)
    res = {"workload": "16 resident geometries (spheres, ellipsoids, tori; %d-%d sources), Poisson "
                       "arrivals, Laplace FP64 / mixed or Helmholtz k in {1,5,10}, SLP, p in {5,9,12}"
                       % (min(g.n_src for g in geoms), max(g.n_src for g in geoms)),
           "policy": "size priority" if size_priority else "fifo", "laplace_fp64_path": laplace_fp64_path,
           "offered": first}
    capacity = first["achieved_req_per_s"]
    saturated = first["span_s"] > 1.15 * first["submit_s"]
    res["saturated_at_offered_rate"] = bool(saturated)
    if saturated:
        res["sustainable"] = phase(0.8 * capacity, duration_s)
    st = srv.stats()
    res["plans_resident"] = st["plans_resident"]
    res["resident_bytes"] = st["resident_bytes"]
    srv.close()
    return res


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
    measure_peaks(pkg, local_rank, torch.cuda.get_device_properties(dev).multi_processor_count)
    if args.only:
        flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
        steps = max(3, args.steps // 2)
        if args.only == "serving":
            res = {"fifo": leg_serving(pkg), "size_priority": leg_serving(pkg, size_priority=True)}
        elif args.only == "target_derivative":
            g, mu = workload()
            res = leg_target_derivative(pkg, torch, dev, g, mu, steps, args.warmup, flush)
        elif args.only == "multi_density":
            g, mu = workload()
            res = leg_multi_density(pkg, torch, dev, g, steps, args.warmup, flush)
        else:
            fn = {"batched": leg_batched, "helmholtz": leg_helmholtz, "sphere": leg_sphere,
                  "conventional": leg_conventional, "lists": leg_lists}[args.only]
            res = fn(pkg, torch, dev, steps, args.warmup, flush)
        if rank == 0:
            print(json.dumps({"leg": args.only, **res}), flush=True)
        return

    g, mu = workload()
    if world > 1:    # each rank evaluates its own density (independent matvec)
        mu = mu * (1.0 + 0.01 * rank)
    precisions = ("fp64", "mixed", "df64")
    plans = {prec: pkg.Plan(g, "laplace", ("slp", "dlp"), p=P, precision=prec, device=local_rank)
             for prec in precisions}
    dmu = torch.from_numpy(mu).to(dev)
    torch.cuda.synchronize()
    tuning = {}
    for prec, pl in plans.items():
        tuning[prec] = pl.autotune(dmu, repeats=3) if not args.no_autotune else pl.get_tuning()
    info = plans["fp64"].info()
    pair_terms = info["n_pair_terms"]
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
        for prec in precisions:
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
    for prec in precisions:
        step_ms, kern_ms = res[prec]
        t_step = agg(step_ms)
        t_kern = agg(kern_ms)
        value = pair_terms * args.steps * world / t_step
        kavg = t_kern / args.steps
        if prec == "df64":
            # double-float on the FP32 pipes: its own FP32 flops against the
            # FP32 peak; the FP64-equivalent rate is kept beside it
            fl = df64_fp32_flops_per_pair(P)
            rf = roofline(fl * info["n_pairs"], kavg, "fp32", ("laplace", prec, "slp+dlp"))
            fe = flops_per_pair(P, "fp64") * info["n_pairs"] / kavg / 1e12
            rf["fp64_equivalent"] = {"flops_per_pair": flops_per_pair(P, "fp64"), "achieved": fe,
                                     "times_fp64_peak": fe / (PEAKS or derived_peaks(152))["fp64"]}
        else:
            fl = flops_per_pair(P, prec)
            rf = roofline(fl * info["n_pairs"], kavg, "fp64" if prec == "fp64" else "fp32",
                          ("laplace", prec, "slp+dlp"))
            # the same launch counted with the a priori per-pair estimate
            sf = a_priori_flops_per_pair(P) + (flops_per_pair(P, prec) - flops_per_pair(P, "fp64"))
            sa = sf * info["n_pairs"] / kavg / 1e12
            rf["a_priori_count"] = {"flops_per_pair": sf, "achieved": sa, "frac": sa / rf["peak"]}
        rf["flops_per_pair"] = fl
        summary[prec] = {"value": value, "ms_per_step": 1e3 * t_step / args.steps,
                         "kernel_ms": 1e3 * kavg, "roofline": rf,
                         "pairs_per_s": info["n_pairs"] * args.steps * world / t_step}

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

    extras = {}
    if not args.no_extras and rank == 0:
        # the oracle beside the Helmholtz and sphere legs: one-GPU runs only
        leg_cpu_s = 0.0 if (args.no_cpu or world != 1) else min(5.0, args.cpu_seconds)
        for name, fn in (("batched", leg_batched), ("helmholtz", leg_helmholtz), ("sphere", leg_sphere),
                         ("conventional", leg_conventional), ("lists", leg_lists)):
            kw = ({"cpu_seconds": leg_cpu_s} if name in ("helmholtz", "sphere")
                  else {"check_targets": 300 if leg_cpu_s > 0 else 0} if name in ("batched", "conventional")
                  else {})
            extras[name] = fn(pkg, torch, dev, max(3, args.steps // 2), args.warmup, flush, **kw)
        extras["helmholtz"].pop("_sample", None)
        extras["target_derivative"] = leg_target_derivative(pkg, torch, dev, g, mu, max(3, args.steps // 2),
                                                            args.warmup, flush,
                                                            check_targets=600 if leg_cpu_s > 0 else 0)
        extras["multi_density"] = leg_multi_density(pkg, torch, dev, g, max(3, args.steps // 2), args.warmup, flush)
        extras["serving"] = leg_serving(pkg)
        extras["serving_size_priority"] = leg_serving(pkg, size_priority=True)

    if rank != 0:
        return
    # ---- CPU baseline (oracle on a bounded sample) + error of both GPU paths
    # there; on rank 0 of a one-GPU run only
    cpu = None
    err = {}
    if not args.no_cpu and world == 1:
        cs = cpu_sample(g, mu, args.cpu_seconds)
        cpu = {"value": cs["value"], "unit": UNIT, "cores": cs["cores"], "kind": "oracle", **host_cpu(),
               "sample": f"{len(cs['idx'])} random targets ({cs['pairs']} pairs, "
                         f"{cs['seconds']:.1f} s) of the benchmark workload, SLP+DLP p=9",
               "single_core": {"value": cs["single_core"]["value"], "unit": UNIT,
                               "sample": f"{cs['single_core']['targets']} of the same targets, "
                                         f"{cs['single_core']['seconds']:.1f} s"}}
        for prec in precisions:
            for l in ("slp", "dlp"):
                got = outs[prec][l].cpu().numpy()[cs["idx"]]
                ref = cs["ref"][l]
                err[f"{prec}_{l}"] = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
        for l in ("slp", "dlp"):
            ref = cs["ref"][l]
            err[f"e2e_fp64_{l}"] = float(np.max(np.abs(host_out[l][cs["idx"]] - ref)) / np.max(np.abs(ref)))

    f = summary["fp64"]
    full = {
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
        "pairs_per_s": f["pairs_per_s"],
        "mixed": {"value": summary["mixed"]["value"], "unit": UNIT, "dtype": "f32 recurrence, f64 sums",
                  "ms_per_step": summary["mixed"]["ms_per_step"], "kernel_ms": summary["mixed"]["kernel_ms"],
                  "roofline": summary["mixed"]["roofline"], "pairs_per_s": summary["mixed"]["pairs_per_s"],
                  "speedup_vs_fp64": summary["mixed"]["value"] / f["value"]},
        "df64": {"value": summary["df64"]["value"], "unit": UNIT,
                 "dtype": "double-float (f32 pairs), f64 geometry offsets and sums",
                 "ms_per_step": summary["df64"]["ms_per_step"], "kernel_ms": summary["df64"]["kernel_ms"],
                 "roofline": summary["df64"]["roofline"], "pairs_per_s": summary["df64"]["pairs_per_s"],
                 "speedup_vs_fp64": summary["df64"]["value"] / f["value"]},
        "error_vs_oracle": err or None,
        "e2e": e2e,
        "gpu_launches": args.steps * sum(pl.info()["launches_per_eval"] for pl in plans.values()),
        "tuning": tuning,
        "clocks": clocks,
        "wall_s_timed_region": wall_s,
        "cpu_baseline": cpu,
        "peaks": PEAKS,
    }
    full.update(extras)
    emit(full, args.detail)
    for p_ in plans.values():
        p_.close()


def _sig(x, digits=4):
    """x rounded to `digits` significant digits (numbers only)."""
    if isinstance(x, bool) or not isinstance(x, float):
        return x
    if x == 0.0 or x != x or x in (float("inf"), float("-inf")):
        return x
    return float(f"{x:.{digits - 1}e}")


def _pick(d, *keys):
    """The listed keys of dict d that exist, floats rounded."""
    return {k: _sig(d[k]) for k in keys if isinstance(d, dict) and k in d}


def _short_roofline(rf):
    out = _pick(rf, "bound", "achieved", "peak", "unit", "frac", "traffic", "pipe", "flops_per_pair")
    src = str(rf.get("peak_source", ""))
    out["peak_source"] = "measured" if src.startswith("measured") else "derived"
    if "a_priori_count" in rf:
        out["a_priori"] = _pick(rf["a_priori_count"], "flops_per_pair", "frac")
    if "fp64_equivalent" in rf:
        out["fp64_equiv"] = _pick(rf["fp64_equivalent"], "achieved", "times_fp64_peak")
    return out


def headline(full, detail_path=None):
    """The last stdout line: the contract's keys with the headline workload's
    numbers, one short block per precision and per secondary workload, all
    floats to four significant digits; everything else goes to the detail
    file.  Kept under HEADLINE_MAX_BYTES."""
    err = full.get("error_vs_oracle") or {}
    line = {k: _sig(full[k]) for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                                       "higher_is_better", "scaling", "vs_baseline", "dtype", "data")}
    cfg = full.get("config", {})
    line["config"] = {"workload": cfg.get("workload"), "n_pairs": cfg.get("n_pairs"),
                      "l2": "flushed between steps"}
    line["roofline"] = _short_roofline(full["roofline"])
    line["kernel_ms"] = _sig(full["kernel_ms"])
    line["error_vs_oracle"] = {k: _sig(v, 2) for k, v in err.items() if k.startswith("fp64")} or None
    for prec in ("mixed", "df64"):
        if prec in full:
            b = full[prec]
            line[prec] = dict(_pick(b, "value", "ms_per_step", "kernel_ms"),
                              frac=_sig(b["roofline"]["frac"]),
                              error={k[len(prec) + 1:]: _sig(v, 2) for k, v in err.items()
                                     if k.startswith(prec + "_")} or None)
    if full.get("e2e"):
        line["e2e"] = _pick(full["e2e"], "value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")
    if full.get("cpu_baseline"):
        line["cpu_baseline"] = _pick(full["cpu_baseline"], "value", "unit", "cores", "kind")
        line["cpu_baseline"]["sample"] = str(full["cpu_baseline"].get("sample", ""))[:60]
    line["gpu_launches"] = full.get("gpu_launches")
    if full.get("clocks"):
        line["clocks"] = _pick(full["clocks"], "sm_mhz", "sm_max_mhz", "reasons")
    legs = {}
    for name in ("helmholtz", "batched", "sphere"):
        if name in full and isinstance(full[name], dict):
            b = full[name]
            sub = b.get("slp", b)                  # Helmholtz: its single-layer plan
            legs[name] = dict(_pick(b, "value"), **_pick(sub, "ms_per_step"),
                              frac=_sig(sub.get("roofline", {}).get("frac")))
            e = sub.get("error_vs_oracle", b.get("error_vs_oracle"))
            if isinstance(e, dict) and "slp" in e:
                legs[name]["err"] = _sig(e["slp"], 2)
    td = full.get("target_derivative")
    if isinstance(td, dict) and isinstance(td.get("mixed"), dict):
        e = td["mixed"].get("error_vs_oracle") or {}
        legs["sp_mixed"] = dict(_pick(td["mixed"], "value"), err=_sig(e.get("sp"), 2))
    srv = full.get("serving")
    if isinstance(srv, dict) and "offered" in srv:
        o = srv["offered"]
        legs["serving"] = dict(_pick(o, "offered_req_per_s", "achieved_req_per_s", "p50_ms", "p99_ms"),
                               saturated=srv.get("saturated_at_offered_rate"))
        if "sustainable" in srv:
            legs["serving"]["at80"] = _pick(srv["sustainable"], "offered_req_per_s", "p50_ms", "p99_ms")
    if legs:
        line["legs"] = legs
    if detail_path:
        line["detail"] = os.path.basename(detail_path)
    text = json.dumps(line, separators=(",", ":"))
    if len(text) > HEADLINE_MAX_BYTES:          # drop the secondary blocks first
        for k in ("legs", "df64", "clocks"):
            line.pop(k, None)
            text = json.dumps(line, separators=(",", ":"))
            if len(text) <= HEADLINE_MAX_BYTES:
                break
    return text


def emit(full, detail_path):
    """Write every number to the detail file, then print the headline as the
    only stdout line."""
    if detail_path:
        d = os.path.dirname(os.path.abspath(detail_path))
        os.makedirs(d, exist_ok=True)
        with open(detail_path, "w") as fh:
            json.dump(full, fh, indent=1)
    print(headline(full, detail_path), flush=True)


if __name__ == "__main__":
    main()
