"""Host-side logic of bench.py on the CPU: the reference arm's JSON line (the oracle on the host
cores; the same contract as the GPU arm's line), the rule that a recorded ncu traffic figure is
reported only while the kernel's sources are unchanged, and the MUFU-bound fraction."""
import argparse
import json
import os
import shutil

import pytest

import bench


def test_reference_arm_prints_one_contract_line(capsys, monkeypatch):
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(gpus=1, steps=2, warmup=3, workload="plain2000x1000")
    bench.run_reference(args, bench.workload("plain2000x1000"), budget_s=0.05)
    lines = [x for x in capsys.readouterr().out.splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["unit"] == "cell-updates/s" and line["higher_is_better"] is True
    assert line["config"]["workload"] == "plain2000x1000"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "consumers" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, workload="plain2000x1000")
    bench.run_reference(args, bench.workload("plain2000x1000"), budget_s=0.05)
    assert capsys.readouterr().out.strip() == ""


def test_recorded_traffic_only_while_the_kernel_sources_are_unchanged(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    kernel, entry = next(iter(rec.items()))
    assert bench.recorded_traffic(kernel) == entry["dram_bytes_per_launch"]
    assert bench.recorded_traffic("no such kernel") is None
    # a copy of the recorded sources with one of them changed: the figure is withdrawn
    for src in entry["sources"]:
        path = src.partition("#")[0]
        os.makedirs(tmp_path / os.path.dirname(path), exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, path), tmp_path / path)
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(kernel) == entry["dram_bytes_per_launch"]
    first = tmp_path / entry["sources"][0].partition("#")[0]
    first.write_bytes(first.read_bytes() + b"\n// changed\n")
    assert bench.recorded_traffic(kernel) is None


def test_mufu_fraction():
    # (1 + 2/m) MUFU operations per cell-update: 10^12 cell-updates at m = 2 take 2 s at 10^12 /s
    assert bench.mufu_frac(1e12, 2, 2000.0, 1e12) == pytest.approx(1.0)
    assert bench.mufu_frac(1e12, 2, 4000.0, 1e12) == pytest.approx(0.5)
