"""Host-side checks of the benchmark's contract that need no GPU: the
profile figures it reports are taken only from a summary made on the
current kernel source, and the reference arm (the oracle on the host
cores) prints the contract's JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _summary(path, digest, traffic=123456789.0):
    with open(path, "w") as f:
        f.write(f"# test summary\n\ntraffic_bytes_per_launch: {traffic:.0f}\nkernel_source_sha256_16: {digest}\n")


def test_profile_figures_follow_the_kernel_source(tmp_path, monkeypatch):
    """A summary carrying the current source hash gives its traffic figure;
    one taken on another source gives none (the bench then reports null)."""
    path = str(tmp_path / "summary.md")
    monkeypatch.setattr(bench, "profile_md", lambda precision, workload="production": path)
    _summary(path, bench.kernel_source_hash("f32"))
    assert bench.profiled("f32", "precision", "traffic_bytes_per_launch") == 123456789.0
    _summary(path, "0" * 16)
    assert bench.profiled("f32", "precision", "traffic_bytes_per_launch") is None
    assert bench.profiled("f32", "no such workload", "traffic_bytes_per_launch") is None


def test_kernel_source_hash_depends_on_the_precision_unit():
    assert bench.kernel_source_hash("f32") != bench.kernel_source_hash("f64")
    assert bench.kernel_source_hash("f32") == bench.kernel_source_hash("f32")


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on a bounded sample of the
    default workload and prints one JSON line with the contract's keys."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == "MLUPS"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_warmup_below_three_is_refused():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode != 0
