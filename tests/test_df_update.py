"""Fast mode's looper update in double-float arithmetic on the FP32 pipe
(the gain and covariance update of the final fit for low-pT loopers) against
strict mode's FP64 update and a long double evaluation of the same formulas,
on 640,000 updates drawn from a Kalman filter run with |q/pT| up to 20
(no GPU needed: the header is compiled for the host)."""
from __future__ import annotations

import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_double_float_update_rounds_like_the_fp64_update(tmp_path):
    exe = tmp_path / "df_update"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off",
                           "-I", os.path.join(ROOT, "paper_2601_20569_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "cpp", "df_update.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr
    print(out.stdout)
    f = out.stdout.split()
    v = {f[i]: float(f[i + 1]) for i in range(len(f) - 1)
         if f[i] in ("df_vs_fp64_mismatch", "df_max_ulps", "fp32_max_ulps")}
    # the updates cancel heavily (FP32 is off by thousands of ulps) ...
    assert v["fp32_max_ulps"] > 1e3
    # ... the double-float results are correctly rounded (within half an ulp
    # of the long double result) and equal the FP64 update's, bit for bit,
    # on all but a vanishing fraction of the 12.8 million results
    assert v["df_max_ulps"] <= 0.5 + 1e-6
    assert v["df_vs_fp64_mismatch"] <= 12
