"""The certified FP32 threshold relies on sqrt.approx.f32 being within 2^-22
relative of the correctly rounded square root; measure it on the GPU at every
float of the variance range the kernels can produce."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_sqrt_approx_relative_error_within_assumed_bound(tmp_path, cuda_device):
    exe = tmp_path / "sqrt_bound"
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                           "-include", "cstring", "-o", str(exe),
                           os.path.join(HERE, "cuda", "sqrt_approx_bound.cu")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    worst = float(out.stdout.strip())
    assert 0.0 <= worst <= 2.0 ** -22, worst
