"""The FP64 kernels' exact bit helpers (sign and order tests, frexp, 2^k,
FP32 <-> FP64 conversions on the integer pipe) against CUDA's own
conversions, frexp and ldexp on every input class of their domains: a
small CUDA program (tests/cuda/f64_helpers_check.cu) built for sm_103a and
run on the GPU."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(d):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = os.path.join(d, "f64_helpers_check")
    subprocess.check_call([nvcc, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-fmad=false",
                           "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_2302_13590_gb300", "csrc"),
                           os.path.join(ROOT, "tests", "cuda", "f64_helpers_check.cu"), "-o", exe])
    return exe


def test_bit_helper_check_builds():
    """The check program cross-compiles for sm_103a (no GPU needed)."""
    with tempfile.TemporaryDirectory() as d:
        assert os.path.exists(_build(d))


@pytest.mark.gpu
def test_bit_helpers_match_cuda_conversions():
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        print(r.stdout.strip())
        assert r.returncode == 0, r.stdout + r.stderr
