"""The integer float<->double conversions used by the final fit's FP64 looper
update (they keep conversions off GB300's narrow FP64 unit) are exact: the
header is compiled for the host and checked against the host's IEEE
conversions on every float bit pattern, 2e8 random doubles and constructed
rounding ties (no GPU needed)."""
from __future__ import annotations

import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_widen_and_narrow_are_exact(tmp_path):
    exe = tmp_path / "fp64_conversions"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_2601_20569_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "fp64_conversions.cpp"),
                           "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    assert " 0 mismatches" in out.stdout
