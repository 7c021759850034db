"""bench.py's contract on CPU: the reference arm (the FP64 oracle timed on the host cores)
prints one JSON line with the keys the driver reads, and the source hash that keys the
recorded DRAM traffic ignores comments and whitespace but not code."""
import io
import json
import os
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import bench


def test_reference_arm_prints_one_contract_line(monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    args = SimpleNamespace(small=True, steps=1, warmup=1, gpus=1)
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.reference_arm(args) == 0
    lines = [l for l in out.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    for k in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.reference_arm(SimpleNamespace(small=True, steps=1, warmup=1, gpus=2)) == 0
    assert out.getvalue().strip() == ""


def test_source_hash_ignores_comments_and_whitespace(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("int f(int x) {\n    return x + 1;  // add one\n}\n")
    b.write_text("// a comment line\nint f(int x) {   return x + 1; }\n")
    c.write_text("int f(int x) {\n    return x + 2;\n}\n")
    assert bench.file_hash(str(a)) == bench.file_hash(str(b))
    assert bench.file_hash(str(a)) != bench.file_hash(str(c))


def test_default_run_is_the_thick_headline_with_extra_legs():
    """With no flags the bench times the thick-sample workload (the largest single-GPU
    configuration) with at least 3 warm-up steps, and adds the other workloads as extra keys."""
    args = bench.parse([])
    assert args.workload == "thick" and args.extras and not args.small
    assert args.warmup >= 3 and args.steps >= 1 and args.gpus == 1
    name, spec, B = bench.thick_spec(False)
    assert (spec.P, spec.Kx, spec.T, spec.Nw, B) == (256, 256, 8192, 1000, 32)
    assert spec.full_grid == (1024, 1024) and spec.roi_origin == (384, 384)
    assert set(bench.LEGS) == {"realistic", "batched", "diff", "thick_pipelined"}


def test_standalone_line_carries_the_contract_keys():
    """--workload realistic|batched|diff prints its leg as a line with the driver's keys."""
    args = bench.parse(["--workload", "diff", "--steps", "4", "--warmup", "3"])
    ctx = SimpleNamespace(world=1)
    leg = {"workload": "diff-P8-K128-T512-W200", "value": 1.0e12, "unit": bench.UNIT, "ms_per_step": 5.0,
           "dtype": "f32", "config": {"probes": 8}, "clocks": {"sm_mhz": 2070.0}, "gpu_launches": 8,
           "roofline": {"bound": "alu", "frac": 0.5}, "rel_l2_err_grad_vs_fp64": 1e-6}
    line = bench.standalone_line(ctx, args, leg)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "clocks", "gpu_launches", "roofline", "e2e",
              "cpu_baseline"):
        assert k in line, k
    assert line["config"]["workload"] == leg["workload"] and line["steps"] == 4
    assert line["rel_l2_err_grad_vs_fp64"] == 1e-6 and line["higher_is_better"] is True
    json.dumps(line)
