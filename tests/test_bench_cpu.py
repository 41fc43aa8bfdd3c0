"""bench.py's host side on CPU: the reference arm's JSON line (the oracle
timed on the host cores), and the counts behind the roofline figures, pinned
to the paper's Table 1 byte counts and to direct element counts."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GDOF/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["E"] == 32768 and d["config"]["N"] == 7
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("N", [1, 3, 7, 15])
def test_algorithmic_bytes_are_table_1(N):
    """Bytes per element: BP1.0 reads q and wJ and writes Mq, BP3.5 reads q
    and 7 factors per GLL node and writes Aq, BP3.0 reads q and 7 factors
    per Gauss point and writes Aq, 8 bytes each; per DOF at N = 7 these
    are 27.4, 72 and 95.7 bytes."""
    n, m = N + 1, N + 2
    _, _, b = bench.alg_counts(N)
    assert b["bp1"] == 8 * (2 * n ** 3 + m ** 3)
    assert b["bp35"] == 8 * 9 * n ** 3
    assert b["bp30"] == 8 * (2 * n ** 3 + 7 * m ** 3)
    if N == 7:
        assert round(b["bp1"] / n ** 3, 1) == 27.4 and b["bp35"] / n ** 3 == 72 and round(b["bp30"] / n ** 3, 1) == 95.7


def _eo_direct(P, Q, sig):
    """Instruction count of an even-odd folded line by brute force: walk the
    folded evaluation one operation at a time."""
    hq, hp = Q // 2, P // 2
    ops = 2 * hq  # x_i + x_{Q-1-i} and x_i - x_{Q-1-i}
    for _ in range(hp):  # each output pair: even and odd dot products, then sum and difference
        even = hq + (1 if Q % 2 else 0)
        odd = hq
        ops += even + odd + 2
    if P % 2:  # the middle output uses one half only (plus the middle input for the even half)
        ops += hq + (1 if (Q % 2 and sig > 0) else 0)
    return ops


@pytest.mark.parametrize("P,Q,sig", [(9, 8, 1), (8, 9, 1), (8, 8, -1), (9, 9, -1), (5, 4, 1), (2, 2, -1), (17, 16, 1)])
def test_even_odd_instruction_count(P, Q, sig):
    inst, flops = bench.eo_cost(P, Q, sig)
    assert inst == _eo_direct(P, Q, sig)
    if min(P, Q) >= 4:
        assert inst < P * Q  # folding beats the direct P*Q multiply-adds (not on 2-point lines)
    assert flops > inst  # every FMA counts two flops


def test_direct_flop_counts():
    """The direct sum-factorisation flop counts at N = 7 by element: three
    interpolation and three projection contractions, 3x3 chain rule, the
    lambda term, six derivative contractions (multiply-add = 2 flops)."""
    N = 7
    n, m = N + 1, N + 2
    std, _, _ = bench.alg_counts(N)
    contract = lambda rows, cols, lines: 2 * rows * cols * lines
    interp = contract(m, n, n * n) + contract(m, n, m * n) + contract(m, n, m * m)
    assert std["bp1"] == 2 * interp + m ** 3
    deriv_gll = 3 * contract(n, n, n * n)
    assert std["bp35"] == 2 * deriv_gll + 18 * n ** 3
    deriv_gauss = 3 * contract(m, m, m * m)
    assert std["bp30"] == 2 * interp + 2 * deriv_gauss + 18 * m ** 3
    # BP1.0 and BP3.0 in one pass share the interpolation
    assert std["bp1_bp30"] == std["bp1"] + std["bp30"] - interp
    _, inst, byts = bench.alg_counts(N)
    assert inst["bp1_bp30"] < inst["bp1"] + inst["bp30"]
    assert byts["bp1_bp30"] == byts["bp1"] + byts["bp30"] - 8 * (n ** 3 + m ** 3)  # q and wJ read once


def test_parse_degrees():
    assert bench.parse_degrees("1-3,7, 11") == [1, 2, 3, 7, 11]
    assert bench.parse_degrees("") == []
