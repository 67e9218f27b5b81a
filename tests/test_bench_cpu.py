"""The host-side parts of bench.py: the reference arm's JSON line and the
oracle samples behind cpu_baseline, for every workload option (run here on a
16^3 sample so that the suite stays fast)."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the contract's keys, the reference
    marked, the cpu_baseline and e2e of the same run, and value > 0."""
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "REF_EDGE", 16)

    class Args:
        steps, warmup, gpus = 2, 1, 1

    assert bench.run_reference(Args()) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.parametrize("kind,density,gravity,phase", [
    ("hit", None, None, "lb"), ("hit", (1.0, 0.1, 0.51, 0.55), None, "lb"),
    ("hit", (1.0, 0.1, 0.51, 0.55), (0.0, 0.0, -1e-5), "lb"), ("droplet", None, None, "lb"),
    ("abc", None, None, "lb"), ("hit", None, None, "weno5"), ("droplet", None, None, "weno5")])
def test_cpu_baseline_samples(monkeypatch, kind, density, gravity, phase):
    """Every workload option gives a positive oracle rate, the thread count it
    used, and a sample description naming the options."""
    monkeypatch.setattr(bench, "SAMPLE_EDGE", 16)
    monkeypatch.setattr(bench, "SAMPLE_STEPS", 2)
    c = bench.cpu_baseline_sample(kind, density, gravity, phase)
    assert c["kind"] == "oracle" and c["unit"] == "MLUPS" and c["value"] > 0 and c["cores"] >= 1
    assert "16^3" in c["sample"]
    if kind == "abc":
        assert "ABC" in c["sample"]
    elif kind == "droplet":
        assert "density ratio 100" in c["sample"]
    if density:
        assert "density contrasts" in c["sample"]
    if gravity:
        assert "buoyancy" in c["sample"]
    if phase == "weno5":
        assert "WENO-5" in c["sample"]


@pytest.mark.parametrize("workload", ["hit", "droplet", "abc", "ensemble"])
def test_reference_arm_follows_the_workload_option(monkeypatch, capsys, workload):
    """The reference arm times the oracle on a sample of the workload the GPU
    arm runs (the ensemble's on the bubbly sample)."""
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "REF_EDGE", 16)

    class Args:
        steps, warmup, gpus, density, gravity, phase = 1, 1, 1, None, None, "lb"

    Args.workload = workload
    assert bench.run_reference(Args()) == 0
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    want = {"hit": "bubbly", "ensemble": "bubbly", "droplet": "droplet", "abc": "ABC"}[workload]
    assert want in d["config"]["workload"]


def test_gravity_argument_takes_three_components():
    """--gravity takes one comma-separated triple (a leading minus in
    scientific notation would read as an option otherwise)."""
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gravity", "0,0"],
                       capture_output=True, text=True)
    assert r.returncode != 0 and "three comma-separated" in r.stderr


def test_reference_arm_from_the_command_line():
    """`python bench.py --impl reference` (the driver's command) prints exactly
    one JSON line with the reference marked, on the default 64^3 sample."""
    import subprocess

    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["warmup"] == 3 and d["steps"] == 1 and d["value"] > 0
    assert "64^3 sample" in d["config"]["workload"]


def test_oracle_references_of_the_error_cases(monkeypatch):
    """The oracle runs behind the default line's errors and CPU baseline: K and
    Phi at every sample, the final fields, a finite droplet pressure jump of
    the right sign (the droplet is at higher pressure), and the stepping time
    counted over both cases."""
    monkeypatch.setattr(bench, "SURR_EDGE", 16)
    monkeypatch.setattr(bench, "SURR_STEPS", 4)
    monkeypatch.setattr(bench, "SURR_EVERY", 2)
    monkeypatch.setattr(bench, "LAP_SAMPLES", [1, 2])
    ref = bench.oracle_references("hit512")
    assert len(ref["K"]) == 2 and len(ref["Phi"]) == 2 and all(k > 0 for k in ref["K"])
    assert len(ref["final"]) == 3 and ref["final"][1].shape == (3, 16, 16, 16)
    assert ref["dp"] > 0 and ref["time_s"] > 0 and ref["cores"] >= 1
    assert ref["updates"] == 16 ** 3 * 4 + bench.LAP_EDGE ** 3 * 2


def test_laplace_jump_of_a_uniform_pressure_is_zero():
    rho = np.ones((32, 32, 32))
    assert bench.laplace_dp(rho, 32, 8.0, 3.0) == 0.0
    rho[:] = 1.0
    z, y, x = np.meshgrid(*[np.arange(32)] * 3, indexing="ij")
    c = 15.5
    inside = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2) < 2.0
    rho[inside] = 1.03
    assert abs(bench.laplace_dp(rho, 32, 8.0, 3.0) - 0.01) < 1e-12
