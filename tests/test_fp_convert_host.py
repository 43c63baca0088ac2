"""The integer float<->double conversions of the refinement kernels, checked
on the host against the host compiler's IEEE-754 conversions.

fp_convert.cuh is plain header code that compiles for the host as well; a
small C++ program (tests/native/fp_convert_check.cpp) runs about 230 million
cases — strided over every float bit pattern, all subnormals near both ends,
exact float midpoints and their double neighbours, the overflow and underflow
edges — and requires identical bits (NaN for NaN)."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_conversions_match_ieee(tmp_path):
    exe = tmp_path / "fp_convert_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", str(ROOT / "paper_2310_16214_gb300" / "csrc"),
                    str(ROOT / "tests" / "native" / "fp_convert_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    assert out.stdout.startswith("OK"), out.stdout
