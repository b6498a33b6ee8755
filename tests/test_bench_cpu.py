"""The benchmark's host-side contract, without a GPU: the reference arm (the
C oracle on the host cores) prints one JSON line with the contract's keys,
non-zero ranks stay silent, the warm-up floor is enforced, and the
algorithmic byte counts behind every roofline fraction equal the per-
subcarrier figures written out by hand from the array sizes."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def run_bench(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=timeout)


@pytest.mark.parametrize("b,u,t,q,expect", [
    (128, 8, 14, 6, 8192 + 14336 + 896 + 2688),   # the metric configuration
    (128, 8, 1, 6, 8192 + 1024 + 64 + 192),       # same, one symbol
    (32, 8, 1, 4, 2048 + 256 + 64 + 128),         # 32x8 16-QAM, one symbol
    (256, 16, 14, 6, 32768 + 28672 + 1792 + 5376),
])
def test_algorithmic_bytes_per_subcarrier(b, u, t, q, expect):
    """H (8BU) + Y (8TB) read once, xhat (8TU) and LLRs (4TUQ) written once."""
    assert bench.algorithmic_bytes_per_sc(b, u, t, q) == expect


def test_algorithmic_bytes_of_16bit_storage():
    # 4-byte complex entries for H and Y, float32 outputs
    assert bench.algorithmic_bytes_per_sc_stored(256, 16, 14, 6, 4) == 16384 + 14336 + 1792 + 5376
    assert bench.algorithmic_bytes_per_sc_stored(128, 8, 14, 6, 8) == bench.algorithmic_bytes_per_sc()


def test_reference_arm_prints_the_contract_line():
    r = run_bench(["--impl", "reference", "--steps", "3", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "Gb/s" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 3 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["subcarriers_per_step"] == bench.NSC_FRAME * bench.FRAMES


def test_reference_arm_is_silent_on_other_ranks():
    r = run_bench(["--impl", "reference", "--steps", "3", "--warmup", "3"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_floor_is_enforced():
    r = run_bench(["--impl", "reference", "--steps", "3", "--warmup", "2"])
    assert r.returncode != 0 and "warmup" in r.stderr


def test_cpu_baseline_line_reports_all_oracle_forms():
    import argparse
    line = bench.cpu_baseline_line(argparse.Namespace(cpu_seconds=0.4, mode="box"))
    assert line["kind"] == "oracle" and line["unit"] == "Gb/s" and line["value"] > 0
    assert line["single_core_gbps"] > 0 and line["numpy_oracle_gbps"] > 0
    assert line["cores"] >= 1


def test_recorded_traffic_matches_the_current_kernel_sources():
    """The committed ncu summary of the dominant kernel was taken on the
    sources that are built now (else the bench reports traffic null)."""
    assert bench.recorded_traffic() is not None, (
        "kernel sources changed since the committed profile: retake the ncu capture")


def test_commands_in_profiles_parse():
    """Every bench.py command line quoted in profiles/ is valid for the
    current argument parser."""
    import glob
    import shlex
    found = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            if "python bench.py" not in line:
                continue
            argv = shlex.split(line.split("python bench.py", 1)[1].strip())
            bench.parser().parse_args(argv)
            found += 1
    assert found >= 4


def test_summaries_are_rounded_to_four_digits():
    out = bench._r({"a": 123.456789, "b": [0.000123456, 7], "c": {"d": 1e-9 / 3}, "e": "x"})
    assert out == {"a": 123.5, "b": [0.0001235, 7], "c": {"d": 3.333e-10}, "e": "x"}
