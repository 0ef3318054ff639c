"""The hand-written edge vector-Jacobian products of the adjoint sweep (first-order f-wave
fluctuations, coupled two-layer and one-layer branches), compiled as host code, against
J^T v with J the oracle's dual-number Jacobian of the same fluctuations. Needs nvcc but no
GPU; the adjoint kernel runs this very code per edge."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_edge_vjp_matches_dual_number_jacobian(orc, tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "vjp_host_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-x", "cu", os.path.join(HERE, "vjp_host_check.cu"), "-o", exe, "-ldl"],
                   check=True, capture_output=True)
    res = subprocess.run([exe, orc.build(), "1e-11"], capture_output=True, text=True)
    print(res.stdout)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.count("worst relative error") == 6
