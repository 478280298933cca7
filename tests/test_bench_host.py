"""bench.py parts that run without a GPU: the reference arm (the FP64 oracle
on bounded samples of the benchmark workload) prints one JSON line with the
contract's keys, and the flop counts per pair behind the rooflines."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=900,
                       env=dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4")))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["unit"] == "pair-terms/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "torus 256x96" in d["config"]["workload"]


def test_flop_counts_per_pair():
    sys.path.insert(0, ROOT)
    import bench
    # mixed p = 9 SLP+DLP: the FP64 count plus the float-float geometry and
    # compensated sums (102 flops per pair; FP64 94)
    assert bench.flops_per_pair(9, "mixed") == 102
    assert bench.flops_per_pair(9, "fp64") == 94
    assert bench.flops_per_pair(9, "fp64") < bench.flops_per_pair(9, "mixed")
    # more orders, more work; layers add work
    for prec in ("fp64", "mixed", "df64"):
        assert bench.flops_per_pair(10, prec) > bench.flops_per_pair(9, prec)
        assert bench.flops_per_pair(9, prec, dlp=False) < bench.flops_per_pair(9, prec)
        assert bench.flops_per_pair(9, prec, sp=True) > bench.flops_per_pair(9, prec)
    # Helmholtz p = 12 with Clenshaw sums: 136 (SLP), 344 (SLP+DLP), 459 (+S'), 295 (SLP+S')
    assert bench.helmholtz_flops_per_pair(12) == 132
    assert bench.helmholtz_flops_per_pair(12, dlp=True) == 336
    assert bench.helmholtz_flops_per_pair(12, dlp=True, sp=True) == 448
    assert bench.helmholtz_flops_per_pair(12, sp=True) == 288


def _full_result():
    """A result object shaped like the GPU arm's (every workload present),
    its floats with many digits, as a one-GPU default run produces it."""
    x = 1.2345678901234567
    rf = {"bound": "alu", "achieved": x, "peak": 73.3 * x, "unit": "TFLOP/s", "frac": 0.8 * x, "traffic": 7.5e7,
          "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)", "pipe": "fp64",
          "peak_source": "measured: register-only FMA probe", "flops_per_pair": 101,
          "hbm": {"achieved_gbs": x, "peak_gbs": 6802.4, "frac": x, "peak_source": "measured"},
          "a_priori_count": {"flops_per_pair": 134, "achieved": x, "frac": x}}
    df_rf = dict(rf, pipe="fp32", fp64_equivalent={"flops_per_pair": 101, "achieved": x, "times_fp64_peak": x})
    leg = {"value": 5.7e10 * x, "ms_per_step": 262.4 * x, "kernel_ms": x, "roofline": rf,
           "error_vs_oracle": {"slp": 1e-15 * x, "targets": 900}, "workload": "w" * 120}
    serving = {"workload": "w" * 150, "policy": "fifo",
               "offered": {k: x for k in ("offered_req_per_s", "requests", "submit_s", "p50_ms", "p99_ms",
                                          "mean_ms", "completed", "achieved_req_per_s", "pair_terms_per_s")},
               "saturated_at_offered_rate": True,
               "sustainable": {k: x for k in ("offered_req_per_s", "p50_ms", "p99_ms", "mean_ms")}}
    return {
        "metric": "TSQBX pair-terms/s at Laplace p=9 (single+double layer), FP64 vs mixed", "value": 7.8e10 * x,
        "unit": "pair-terms/s", "n_gpus": 1, "steps": 20, "warmup": 5, "ms_per_step": 49.1 * x,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "torus 256x96 quads, 294912 sources, 589824 targets, octree lists n_max=64, "
                               "Laplace SLP+DLP p=9", "p": 9, "n_pairs": 383389640, "l2": "flushed"},
        "roofline": rf, "kernel_ms": 49.1 * x, "pairs_per_s": x,
        "mixed": {"value": 3.3e12 * x, "ms_per_step": x, "kernel_ms": x, "roofline": dict(rf, pipe="fp32")},
        "df64": {"value": 3.3e11 * x, "ms_per_step": x, "kernel_ms": x, "roofline": df_rf},
        "error_vs_oracle": {f"{p}_{l}": 1e-7 * x for p in ("fp64", "mixed", "df64", "e2e_fp64") for l in ("slp", "dlp")},
        "e2e": {"value": 7.6e10 * x, "unit": "pair-terms/s", "h2d_bytes_per_step": 2359296,
                "d2h_bytes_per_step": 9437188},
        "gpu_launches": 120, "tuning": {"fp64": {"lanes_per_target": 0, "max_item_iters": 0, "kernel_ms": x}},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 400},
        "cpu_baseline": {"value": 3.0e8 * x, "unit": "pair-terms/s", "cores": 16, "kind": "oracle",
                         "cpu_model": "Neoverse-V2", "nproc": 16,
                         "sample": "4321 random targets (2812345 pairs, 12.0 s) of the benchmark workload, SLP+DLP p=9"},
        "peaks": {"fp64": 1.2, "fp32": 77.0, "source": "measured"},
        "helmholtz": {"value": 5.7e10 * x, "slp": leg, "slp+dlp": leg, "slp+dlp+sp": leg, "unit": "pair-terms/s"},
        "batched": leg, "sphere": leg, "conventional": {"cases": [leg] * 10},
        "lists": {"cases": [{"gpu_ms": x, "host_ms": x}] * 3},
        "target_derivative": {"fp64": leg, "mixed": dict(leg, error_vs_oracle={"slp": x, "dlp": x, "sp": 3e-7 * x}),
                              "df64": leg},
        "serving": serving, "serving_size_priority": serving,
    }


def test_gpu_arm_headline_is_short_and_complete(scratch, capsys):
    """The GPU arm's last stdout line (the one a reader of the run's tail
    sees) parses, stays under the size limit with every workload present,
    and carries the contract's keys; the full result goes to the detail file."""
    sys.path.insert(0, ROOT)
    import bench
    full = _full_result()
    detail = str(scratch / "detail.json")
    bench.emit(full, detail)
    out = capsys.readouterr().out.splitlines()
    assert len(out) == 1
    assert len(out[0].encode()) <= bench.HEADLINE_MAX_BYTES < 3000
    d = json.loads(out[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "kernel_ms", "cpu_baseline",
                "e2e", "clocks", "gpu_launches", "mixed", "error_vs_oracle"):
        assert key in d, key
    assert d["value"] > 0 and d["config"]["workload"].startswith("torus 256x96")
    assert d["roofline"]["peak_source"] == "measured" and d["roofline"]["frac"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 16
    assert set(d["mixed"]) >= {"value", "ms_per_step", "frac", "error"}
    assert d["legs"]["serving"]["p99_ms"] > 0
    with open(detail) as fh:
        assert json.load(fh)["conventional"]["cases"][0]["value"] == full["conventional"]["cases"][0]["value"]


def test_df64_and_a_priori_flop_counts():
    sys.path.insert(0, ROOT)
    import bench
    # the a priori estimate: 6p + 20 single layer, + 4 per pair-term + 20 double layer
    assert bench.a_priori_flops_per_pair(9) == 134
    assert bench.a_priori_flops_per_pair(9, dlp=False) == 74
    # double-float FP32 flops per pair at p = 9: 1016 with both layers, 716 single layer, +104 for S'
    assert bench.df64_fp32_flops_per_pair(9) == 1016
    assert bench.df64_fp32_flops_per_pair(9, dlp=False) == 716
    assert bench.df64_fp32_flops_per_pair(9, sp=True) == 1120
    # lambda_n is a float up to n = 12 (its products then take DWTimesFP)
    assert [bench._lambda_is_float(n) for n in (1, 2, 12, 13, 20)] == [True, True, True, False, False]
    # each further order adds one Q' recurrence step: 60 or 62 FP32 flops,
    # plus 2 where the top coefficients stop being floats
    for p in range(3, 21):
        assert bench.df64_fp32_flops_per_pair(p) - bench.df64_fp32_flops_per_pair(p - 1) in (60, 62, 64)
