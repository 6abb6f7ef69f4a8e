"""The BF16 engine's last hidden layer uses tanh x = 1 - 2 / (exp(2x) + 1) with the hardware
exponential (it feeds the FP32 output dot, so it must be accurate where the other layers use
tanh.approx).  Its absolute error against double-precision tanh must stay within a small
multiple of CUDA tanhf's own."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_tanh_out_error(tmp_path):
    exe = str(tmp_path / "tanh_out_check")
    src = os.path.join(HERE, "cuda", "tanh_out_check.cu")
    inc = ["-I", os.path.join(ROOT, "paper_2606_04895_gb300", "csrc"), "-I", os.path.join(ROOT, "include")]
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", *inc, "-o", exe, src],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    ours, ref = (float(v) for v in out.split()[1:3])
    assert ours < 1e-6, out
    assert ours < 4 * ref + 1e-7, out
