"""The step kernels convert between FP64 and FP32 on the integer ALU
(f32_rn, f64_of in step_math.cuh): their results must be the IEEE
conversions bit for bit, or the mixed path would change with them.  The
header's host path is compiled with nvcc and checked against the C casts on
a few million inputs (tests/host/conversion_bits.cu)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_conversions_match_ieee_casts():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "conversion_bits")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_1805_05128_gb300", "csrc"),
                        "-x", "cu", os.path.join(ROOT, "tests", "host", "conversion_bits.cu"), "-o", exe],
                       check=True, capture_output=True, text=True)
        out = subprocess.run([exe, "2000000"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "f32_rn: 0 mismatches" in out.stdout and "f64_of: 0 mismatches" in out.stdout, out.stdout
