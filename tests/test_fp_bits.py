"""The integer-pipe binary32 <-> binary64 conversions used by the pseudo-time
update (csrc/fp_bits.cuh) agree bit for bit with the host's IEEE 754
conversions: exhaustive over binary32 for widening, ties, binade edges and
random operands for narrowing (tests/fp_bits_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2209_04481_gb300", "csrc")


def test_fp_bits_match_host_conversions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "fp_bits_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "fp_bits_check.cpp"),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
