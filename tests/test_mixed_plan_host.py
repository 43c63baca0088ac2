"""The mixed-radix FFT planner (the constexpr plan of fft_mixed.cuh that
every compile-time kernel is built from), checked on the host without a GPU:
tests/native/mixed_plan_check.cu verifies, for all 172 lengths 2^a 3^b 5^c
up to 12288 that are not powers of two, that the radices multiply to n in
the fewest stages possible (against an independent dynamic program), that
every stage fits the block's threads, and that the block fits the hardware
limits."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="needs nvcc")
def test_mixed_radix_plans(tmp_path):
    exe = tmp_path / "mixed_plan_check"
    subprocess.run(["nvcc", "-std=c++17", "--expt-relaxed-constexpr", "-I",
                    str(ROOT / "paper_2310_16214_gb300" / "csrc"),
                    str(ROOT / "tests" / "native" / "mixed_plan_check.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip() == "OK 172", out.stdout
