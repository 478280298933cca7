"""The paper's cost-model arithmetic (Tables 2-3, Sec. 5.2) from the golden
constants: the pair-term unit c_ts (p+1) reproduces the paper's ~9x TSQBX
speedup and its n_mpole ~ 291 estimate."""
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cost_model_table3.txt")


def load():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_tsqbx_speedup_and_nmpole():
    c = load()
    p = 5
    speedup = c["c_p2qbxl"] * (1 + p) ** 2 / (c["c_ts"] * (1 + p))
    assert round(speedup) == c["predicted_ts_speedup_p5"]
    assert speedup == pytest.approx(9.02, abs=0.01)
    pq, pf = 5, 15
    nm = c["c_m2qbxl"] / c["c_ts"] * ((1 + pf) ** 3 + (1 + pq) ** 2 * (1 + pf) + (1 + pq) ** 3) / (1 + pq)
    assert abs(nm - c["nmpole_optimum_5_15"]) < 1.0
