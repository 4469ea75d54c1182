"""Host-side checks of the schedule autotuner's search space and of the
benchmark's reference arm (the oracle on the host cores), which need no GPU."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_autotune_candidates_are_valid_splits():
    from paper_1402_6297_gb300 import autotune
    for knob, values in autotune.KNOBS.items():
        assert values, knob
        if knob.startswith("NFS_N1_"):
            n = int(knob[len("NFS_N1_"):])
            for n1 in values:
                # both factors must be register DFT lengths (divisors of 48)
                assert n % n1 == 0 and 48 % n1 == 0 and 48 % (n // n1) == 0, (knob, n1)


def test_tuning_header_uses_known_knobs():
    from paper_1402_6297_gb300 import autotune
    path = autotune.TUNING_H
    if not os.path.exists(path):
        pytest.skip("no tuning.h")
    lines = open(path).read().splitlines()
    for i, line in enumerate(lines):
        if line.startswith("#define"):
            _, name, value = line.split()
            assert name in autotune.KNOBS and int(value) in autotune.KNOBS[name], line
            # guarded so that command-line settings (the autotuner's variants) win
            assert lines[i - 1] == f"#ifndef {name}", line


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--cpu-seconds", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
