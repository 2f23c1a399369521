"""The integer-pipe binary64 multiply and reciprocal of the CUDA kernels (csrc/hw_fp64_int.h), compiled
for the host: every product the fast path accepts equals the host's IEEE-754 multiply bit for bit, and
it accepts every product of normal operands whose result is normal (the kernels' data), plus signed
zeros; every reciprocal is within one ulp of the host's correctly rounded 1/x, and every operand with
a normal reciprocal is accepted."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2208_01260_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fp64int") / "fp64_int_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I" + CSRC,
                    os.path.join(HERE, "fp64_int_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_integer_multiply_matches_ieee(checker, seed):
    r = subprocess.run([checker, "3000000", str(seed)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    accepted, bad, missed = (int(v) for v in r.stdout.split()[-3:])
    assert bad == 0 and missed == 0
    assert accepted > 2000000


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_reciprocal_within_one_ulp(checker, seed):
    r = subprocess.run([checker, "2000000", str(seed), "rcp"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    accepted, bad, missed = (int(v) for v in r.stdout.split()[-3:])
    assert bad == 0 and missed == 0
    assert accepted > 3000000
