"""The exponent helpers of the fixed-point sketch (exponent bound of a vector
maximum, scaling by a power of two, positivity test) are integer-instruction
rewrites of frexp, ldexp and x > 0.  This compiles their host path with nvcc
and checks them bit for bit against the C library on random doubles,
subnormals and special values (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_exponent_helpers_match_libm(tmp_path):
    exe = nvcc()
    if exe is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path / "exponent_helpers")
    src = os.path.join(HERE, "native", "exponent_helpers.cu")
    res = subprocess.run([exe, "-std=c++17", "-O2", "-o", out, src], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([out], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    checked, bad = (int(v) for v in run.stdout.split()[1::2])
    assert checked > 250000 and bad == 0   # half the random patterns are negative
