"""The integer FP64 -> double-float split used by the GPU kernels (df_split_int in
csrc/df64.cuh) is compiled for the host and checked bit for bit against its
definition, hi = RN_FP32(x) and lo = RN_FP32(x - hi), on random bit patterns
over the handled exponent range [-60, 126] and beyond, plus the ties and
near-ties of the 24-bit rounding and the carries into the next binade."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2209_02815_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_integer_split_matches_fp32_rounding(tmp_path):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path / "df_split_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-I", CSRC,
                    os.path.join(HERE, "native", "df_split_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe, "300000"], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    tried, handled, bad = map(int, r.stdout.split()[-3:])
    assert bad == 0 and handled > 0.8 * tried
