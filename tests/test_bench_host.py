"""Host-side logic of bench.py that needs no GPU: the DRAM traffic scaling and work models of
the roofline objects, the oracle error statement, and the reference arm's JSON line (the CPU
oracle timed on a small workload)."""
import importlib.util
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_dram_traffic_scales_with_units_and_covers_only_captured_shapes():
    b = _bench_module()
    table = b.load_dram_per_unit()
    assert table, "profiles/dram_per_unit.json missing or empty"
    for kernel, e in table.items():
        p, op, prec = e["shape"]
        one = b.dram_traffic(table, kernel, p, op, prec, 1000)
        assert one == pytest.approx(1000 * e["bytes_per_unit"])
        assert b.dram_traffic(table, kernel, p, op, prec, 2000) == pytest.approx(2 * one)
        # another degree, operator or precision: no capture, no figure
        assert b.dram_traffic(table, kernel, p + 1, op, prec, 1) is None
        assert b.dram_traffic(table, kernel, p, "mass" if op == "stiffness" else "stiffness", prec, 1) is None
        assert b.dram_traffic(table, kernel, p, op, "fp64", 1) is None


def test_flop_models():
    """Work models of the roofline numerators: per-piece moment count and the cut-row count."""
    b = _bench_module()
    q, nb = 5, 9
    assert b.moment_flops(4, 10) == 2 * 10 * (nb * q ** 3 + nb * nb * q * q + nb ** 3 * q)
    info = {"cut_gauss_pairs": 1, "box_points_fst": 0, "box_points_st": 0, "box_points_t": 0, "cut_elem_pairs": 0}
    assert b.cutrows_flops(4, True, info) == 2 * 7 * q ** 4
    assert b.cutrows_flops(4, False, info) == 2 * 3 * q ** 4


def test_reference_arm_prints_one_line_with_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n-el", "12", "--p", "2", "--sample-rows", "40"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "nnz/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle-sf" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_row_error_stats_against_the_oracle_rows():
    """The error statement of the bench line: GPU-side values compared row by row with the
    oracle job's rows (here: the oracle's own rows with a planted relative error)."""
    b = _bench_module()
    from oracle.formation import OracleMesh
    from paper_2211_06427_gb300 import synthetic
    desc = synthetic.c1_ball_p2_8()
    om = OracleMesh(desc)
    from oracle.sfrow import RowOracle
    rows = np.sort(np.nonzero(om.geo.fclass != 0)[0][:25])
    ref = RowOracle(om).rows("mass", rows)
    res = {"rows": rows, "lengths": np.array([len(ref[int(i)]) for i in rows]),
           "values": np.concatenate([ref[int(i)] for i in rows]), "n_interior": 0, "n_cut": len(rows)}
    vals = np.zeros(int(om.geo.rowptr[-1]))
    for i in rows:
        vals[om.geo.rowptr[i]:om.geo.rowptr[i + 1]] = ref[int(i)] * (1 + 1e-6)
    st = b.row_error_stats(vals, om.geo.rowptr, res)
    assert st["rows"] == 25 and st["max_row_err"] == pytest.approx(1e-6, rel=1e-6)
