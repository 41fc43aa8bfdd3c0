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


def _fake_run():
    """A full result of the shape run_ours produces (every side section
    filled, a 15-degree sweep of nine operator columns), with made-up
    numbers: what matters here is the size and the keys."""
    col = {"ms": 1.2345678, "gdofs": 12.345678, "alg_gbs": 5432.1, "hbm_frac": 0.8123, "copy_gbs_at_size": 6012.3,
           "copy_frac_at_size": 0.9, "ratio_stream_gbs": 6100.0, "ratio_read_planes": 8, "hbm_bound_gdofs": 80.0,
           "smem_frac": 0.4, "fp64_tflops": 1.1, "fp64_issue_frac": 0.7}
    names = ("bp1", "bp35", "bp30", "bp1_bp30", "bp30_points", "bp35_f32", "bp30_f32", "bp35_f16", "bp30_f16")
    sweep = {"workload": "x" * 300, "copy_roofline": "y" * 150,
             "rows": [dict({"N": N, "dofs": 32768 * (N + 1) ** 3}, **{k: dict(col) for k in names})
                      for N in range(1, 16)]}
    kern = {k: {"ms": 1.0, "gdofs": 10.0, "alg_gbs": 400.0, "hbm_frac": 0.06, "fp64_tflops": 1.3,
                "fp64_frac": 1.05, "fp64_issue_frac": 0.8, "smem_frac": 0.3} for k in bench.KERNELS}
    line = {"metric": bench.METRIC, "value": 4.86123456789, "unit": "GDOF/s", "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 10.3512345, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench.step_config(32768, 7, 1.0, 1),
            "e2e": {"value": 4.8, "unit": "GDOF/s", "h2d_bytes_per_step": 14155776, "d2h_bytes_per_step": 40265728,
                    "ms_per_step": 10.49, "steps": 20, "windows_ms_per_step": [10.4, 10.5, 10.49, 10.6, 10.45],
                    "reported": "median of the five windows", "pipelining": "z" * 200,
                    "outputs_match_device_step": True},
            "gpu_launches": 80,
            "step_unfused": {"ms_per_step": 11.3, "value": 4.4, "unit": "GDOF/s", "steps": 20, "kernels": "k" * 80},
            "roofline": {"kernel": "bp1_bp30", "bound": "alu", "unit": "TFLOP/s", "achieved": 1.326, "peak": 1.259,
                         "frac": 1.05, "peak_source": "p" * 100, "flop_count": "f" * 150, "fp64_issue_frac": 0.8,
                         "fp64_probe_tflops": 1.057, "fp64_issue_frac_of_probe": 0.95, "fp64_probe": "q" * 120,
                         "traffic": 1625391104,
                         "hbm": {"achieved_gbs": 378.0, "peak_gbs": 6780.0, "peak_source": "measured", "frac": 0.056},
                         "smem": {"bytes_per_elem": 100000, "achieved_gbs": 7000.0, "peak_gbs": 40000.0, "frac": 0.2,
                                  "peak_source": "s" * 100}},
            "cpu_baseline": {"value": 0.11, "unit": "GDOF/s", "cores": 16, "kind": "oracle", "sample": "c" * 150,
                             "single_thread": {"value": 0.01, "unit": "GDOF/s", "cores": 1, "sample": "d" * 80},
                             "host": "aarch64, Neoverse-V2"},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "power_w_max": 800.0, "samples": 300, "reasons": []},
            "kernels": kern}
    tight = {"tol": 1e-13}
    for k in ("fp64", "mixed", "mixed16", "mixed_tc"):
        tight[k] = {"solves_per_s": 4.0, "iters": 1000, "outer": 6, "relres": 7e-14, "status": 0,
                    "rel_err_vs_u_I": 2e-12, "rel_diff_vs_fp64_solve": 5e-12}
        tight[k + "_speedup"] = 7.9
    pcg = {"workload": "w" * 200, "tight": tight, "fp64": dict(tight["fp64"])}
    batch = {"workload": "b" * 150, "dofs_per_pass": 10 ** 8, "separate_launches": {"ms": 30.0, "gdofs": 3.0},
             "persistent_default": {"ms": 25.0, "gdofs": 4.0}, "persistent_tuned": {"ms": 20.0, "gdofs": 5.0,
                                                                                     "config": {"threads": 256}},
             "graph": {"ms": 20.0, "gdofs": 5.0}, "tuner_candidates": 32}
    serve = {"workload": "s" * 200,
             "steady_state": {"arrival_rate_per_s": 12.0, "served_per_s": 12.0, "p50_s": 1.0, "p99_s": 3.0,
                              "queue_depth": {"every_0.5s": list(range(60))}},
             "config_arrivals_200_per_s": {"fifo": {"offered_per_s": 200.0, "served_per_s": 15.0, "p50_s": 9.0,
                                                    "p99_s": 19.0}}}
    return line, {"sweep": sweep, "small_case": {"us_per_launch_graph": 3.0}, "pcg": pcg, "batch": batch,
                  "serve": serve}


def test_headline_is_last_and_compact(capsys, tmp_path):
    """The last stdout line carries the contract's keys in a few KB; every
    side section comes before it on a line of its own, and the side file
    holds the full result."""
    line, sections = _fake_run()
    side = tmp_path / "sections.json"
    bench.emit(line, sections, str(side))
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1 + sum(v is not None for v in sections.values())
    head = json.loads(out[-1])
    assert len(out[-1]) <= bench.HEADLINE_MAX_BYTES
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "roofline",
              "cpu_baseline", "clocks"):
        assert k in head, k
    assert head["e2e"]["h2d_bytes_per_step"] == 14155776 and head["e2e"]["d2h_bytes_per_step"] == 40265728
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "fp64_issue_frac"):
        assert k in head["roofline"], k
    assert head["summary"]["pcg_tol_1e-13"]["mixed_tc"]["rel_diff_vs_fp64_solve"] == 5e-12
    assert head["summary"]["serve"]["config"]["offered_per_s"] == 200.0
    assert head["summary"]["serve"]["steady"]["arrival_rate_per_s"] == 12.0
    for ln in out[:-1]:
        assert json.loads(ln)["section"] in sections
    full = json.loads(side.read_text())
    assert len(full["sections"]["sweep"]["rows"]) == 15


def test_bench_defines_each_function_once():
    """A second definition of a function would silently replace the first."""
    import ast
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    names = [n.name for n in tree.body if isinstance(n, (ast.FunctionDef, ast.ClassDef))]
    assert len(names) == len(set(names)), sorted(n for n in names if names.count(n) > 1)
