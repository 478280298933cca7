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
    # compensated sums (109 flops per pair)
    assert bench.flops_per_pair(9, "mixed") == 109
    assert bench.flops_per_pair(9, "fp64") < bench.flops_per_pair(9, "mixed")
    # more orders, more work; layers add work
    for prec in ("fp64", "mixed", "df64"):
        assert bench.flops_per_pair(10, prec) > bench.flops_per_pair(9, prec)
        assert bench.flops_per_pair(9, prec, dlp=False) < bench.flops_per_pair(9, prec)
        assert bench.flops_per_pair(9, prec, sp=True) > bench.flops_per_pair(9, prec)
    # Helmholtz p = 12 with Clenshaw sums: 136 (SLP), 344 (SLP+DLP), 459 (+S'), 295 (SLP+S')
    assert bench.helmholtz_flops_per_pair(12) == 136
    assert bench.helmholtz_flops_per_pair(12, dlp=True) == 344
    assert bench.helmholtz_flops_per_pair(12, dlp=True, sp=True) == 459
    assert bench.helmholtz_flops_per_pair(12, sp=True) == 295
