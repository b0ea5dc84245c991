"""The library's protected division (generated PTX: reciprocal seed, one
Newton step, Markstein's remainder correction, slow path for extreme
operands) equals CUDA's correctly rounded division bit for bit.

This GPU test runs a sample: random bit patterns over every exponent
(zeros, subnormals, infinities and NaN included), random significands under
every one of the 256 x 256 exponent pairs, and 1/64 of all 2^46 significand
pairs in [1, 2).  The full significand sweep is the same program with
`mant -1 64` (see the division profile under profiles/).
"""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    import paper_1601_00221_gb300 as gp
    gp.build.build()
    exe = str(tmp_path_factory.mktemp("div") / "div_check")
    subprocess.check_call([gp.build._nvcc(), *gp.build.ARCH, "-O3", "-std=c++17", "-fmad=false",
                           "-ftz=false", "-prec-div=true", "-I", gp.build.GEN,
                           os.path.join(HERE, "div_check.cu"), "-o", exe])
    return exe


@pytest.mark.parametrize("args", [["rand", "512", "7"], ["exps", "64", "11"], ["mant", "37", "64"]])
def test_division_matches_ieee(checker, args):
    r = subprocess.run([checker, *args], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout
