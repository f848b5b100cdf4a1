"""Host-side logic of bench.py that needs no GPU: the DRAM traffic scaling of the roofline
objects and the reference arm's JSON line (the CPU oracle timed on a small workload)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Args:
    def __init__(self, p, op, prec):
        self.p, self.op, self.prec = p, op, prec


def test_dram_traffic_scales_with_units_and_covers_only_captured_shapes():
    b = _bench_module()
    for kernel, (shape, per_unit, counter, src) in b.DRAM_PER_UNIT.items():
        assert os.path.exists(os.path.join(ROOT, src)), src
        args = _Args(*shape)
        one = b.dram_traffic(kernel, args, {counter: 1000}, None)
        two = b.dram_traffic(kernel, args, {counter: 2000}, None)
        assert one == pytest.approx(1000 * per_unit)
        assert two == pytest.approx(2 * one)
        assert b.dram_traffic(kernel, args, {}, 500) == pytest.approx(500 * per_unit)
        # another degree, operator or precision: no capture, no figure
        assert b.dram_traffic(kernel, _Args(shape[0] + 1, shape[1], shape[2]), {counter: 1}, None) is None
        assert b.dram_traffic(kernel, _Args(shape[0], "mass", shape[2]), {counter: 1}, None) is None
        assert b.dram_traffic(kernel, _Args(shape[0], shape[1], "fp64"), {counter: 1}, None) is None


def test_reference_arm_prints_one_line_with_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n-el", "12", "--p", "2"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "config"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "nnz/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
