"""Host-side logic of bench.py, on the CPU: the reference arm's JSON line (the
oracle timed on the host cores), its silence on ranks other than 0, the
roofline denominators, and the recorded DRAM traffic that goes stale with the
kernel sources."""
import importlib.util
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _run(args, **env):
    e = dict(os.environ)
    e.update(env)
    return subprocess.run([sys.executable, str(ROOT / "bench.py")] + args, env=e, capture_output=True, text=True,
                          timeout=300, cwd=ROOT)


def test_reference_arm_prints_one_oracle_line():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n", "64", "--ref-seconds", "1"])
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "force cells/s" and d["unit"] == "cells/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "uniform-64x64-lognormal-taper"


def test_reference_arm_other_ranks_do_no_work():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n", "64"], RANK="1", WORLD_SIZE="2")
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == ""


def test_peaks_prefer_the_measured_file(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    assert bench.peaks() == (1234.5, "measured")


def test_recorded_traffic_goes_stale_with_the_sources(bench, tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({"csrc_sha256": "abc", "dram_bytes_per_launch": {"col": 123}}))
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "csrc_digest", lambda: "abc")
    assert bench.recorded_traffic("col") == 123
    assert bench.recorded_traffic("row_fwd") is None
    monkeypatch.setattr(bench, "csrc_digest", lambda: "changed")
    assert bench.recorded_traffic("col") is None


def test_committed_traffic_record_names_the_timed_kernels(bench):
    d = json.loads((ROOT / "profiles" / "traffic.json").read_text())
    assert set(d["dram_bytes_per_launch"]) == {"row_fwd", "col", "row_inv"}
    assert d["sources"] == list(bench.KERNEL_SOURCES)
    assert "--clock-control none" in d["command"]


def test_fp32_pipe_record_goes_stale_with_the_sources(bench, tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    rec = {"fma_pipe_active_pct": 48.0, "issue_active_pct": 49.0, "duration_us": 220.0}
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({"csrc_sha256": "abc", "fp32_pipe_per_launch": {"col": rec}}))
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "csrc_digest", lambda: "abc")
    assert bench.recorded_ncu("col", "fp32_pipe_per_launch") == rec
    assert bench.recorded_ncu("row_inv", "fp32_pipe_per_launch") is None
    monkeypatch.setattr(bench, "csrc_digest", lambda: "changed")
    assert bench.recorded_ncu("col", "fp32_pipe_per_launch") is None


def test_committed_records_match_the_sources(bench):
    """The committed DRAM and FP32-pipe record was taken on the kernel sources in
    the tree (else the bench would report it as null)."""
    d = json.loads((ROOT / "profiles" / "traffic.json").read_text())
    assert d["csrc_sha256"] == bench.csrc_digest()
    assert set(d["fp32_pipe_per_launch"]) == {"row_fwd", "col", "row_inv"}


def test_profile_commands_use_flags_bench_accepts():
    """Every bench.py flag a committed profile summary's command uses is one the
    bench's argument parser knows (the summaries must stay runnable)."""
    import re
    helptext = _run(["--help"]).stdout
    flags = set()
    for f in (ROOT / "profiles").glob("*.md"):
        for line in f.read_text().splitlines():
            if "bench.py" in line:
                flags.update(re.findall(r"(--[a-z][a-z0-9-]*)", line.split("bench.py", 1)[1]))
    flags -= {"--clock-control", "--set", "--section", "--metrics", "--csv", "--log-file", "--kernel-name-base"}
    assert flags, "no bench.py command found under profiles/"
    missing = sorted(fl for fl in flags if fl not in helptext)
    assert not missing, missing
