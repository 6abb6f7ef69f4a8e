"""The device Philox4x32-10 that draws every proposal, momentum, accept uniform and tree
direction: its words must equal the published known-answer vectors and cuRAND's
curand_Philox4x32_10 (a separate implementation of the same generator) on 2^20 random
counters and keys."""
import os
import subprocess

import pytest

from test_oracle_rng import kat_vectors

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_device_philox_known_answers_and_curand(tmp_path):
    exe = str(tmp_path / "philox_check")
    src = os.path.join(HERE, "cuda", "philox_check.cu")
    inc = ["-I", os.path.join(ROOT, "paper_2606_04895_gb300", "csrc"), "-I", os.path.join(ROOT, "include")]
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", *inc, "-o", exe, src],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    words = [int(v, 16) for v in out[0].split()[1:]]
    want = [w for _, _, o in kat_vectors() for w in o]
    assert words == want, out[0]
    assert out[1].startswith("mismatches 0 of "), out[1]
