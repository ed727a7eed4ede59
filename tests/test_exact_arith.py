"""The integer forms of the split/merge decisions used by the resampling kernel
(paper_1303_5986_gb300/csrc/we_exact.cuh) against the host's IEEE double arithmetic: fl(w/c)
for every copy count up to 2048 and u < fl(w/(w+q)) for random, equal and adjacent uniforms."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_exact_integer_forms_match_ieee(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "exact_arith_check")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "exact_arith_check.cpp")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok"), out.stdout
