"""The register-resident separable chains' index pattern and arithmetic, on
the CPU (no GPU): tests/host/sep_chain_check.cu includes the CUDA source and
runs its host-compilable step, chain and fused-pair functions against dense
products of the step matrices (see that file's header)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "sep_chain_check.cu")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_register_chain_pattern_and_arithmetic_on_host(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "sep_chain_check")
    inc = os.path.join(HERE, "..", "include")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=compute_103a",
                    "-I", inc, SRC, "-o", exe], check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "pattern mismatches: 0" in r.stdout and "failures: 0" in r.stdout
