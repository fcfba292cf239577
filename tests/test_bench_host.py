"""The benchmark's host side on CPU: the reference arm (the oracle timed on
the host cores) prints one JSON line with the contract's keys, and the native
arm refuses to run without a GPU instead of falling back to the CPU."""
import json
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    out = _run("--impl", "reference", "--steps", "2", "--warmup", "3", "--workload", "2000bus_fp64_adjoint")
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "us/system" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "2000bus_fp64_adjoint" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"].startswith("2 of the 2 requested steps") and "bounded" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_default_workload_is_the_largest_single_gpu_configuration():
    sys.path.insert(0, ROOT)
    import bench
    from kktgen import config_sequence
    assert bench.DEFAULT_WORKLOAD == "70000bus_fp32_refined"
    cfg = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert cfg["fp32"] and cfg["refine"] in ("auto", "fgmres")
    sizes = [config_sequence(c).n for c in (0, 1, 3)]
    assert config_sequence(cfg["cfg"]).n == max(sizes) == 490_000


def test_timing_rules_are_enforced():
    out = _run("--impl", "reference", "--steps", "1", "--warmup", "2")
    assert out.returncode != 0 and "warmup" in (out.stdout + out.stderr)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_native_arm_needs_a_gpu():
    out = _run("--steps", "1", "--warmup", "3", "--no-cpu-baseline", "--no-variants")
    assert out.returncode != 0 and "GPU" in (out.stdout + out.stderr)


def test_reference_arm_of_the_batched_workload():
    out = _run("--impl", "reference", "--steps", "1", "--warmup", "3", "--workload", "10000bus_x64_batched",
               "--ref-budget", "2", "--cpu-budget", "2")
    assert out.returncode == 0, out.stderr
    d = json.loads([l for l in out.stdout.splitlines() if l.strip().startswith("{")][-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["workload"] == "10000bus_x64_batched"
    assert "scenario systems" in d["cpu_baseline"]["sample"]
