"""Host check of the magic-number division used by the LM kernels' index
arithmetic (exact quotient from one multiply-high): compiles
tests/host/divmagic_check.cu as host code with nvcc and runs it (no GPU)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not on PATH")
def test_div_magic_quotients_exact(tmp_path):
    exe = str(tmp_path / "divmagic_check")
    subprocess.run(["nvcc", "-O2", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "host", "divmagic_check.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "bad 0" in out.stdout
