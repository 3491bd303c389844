"""The host-side rules of the batched and TMA forms (tests/host_tables_check.cu), built with nvcc
and run on the CPU: which passes take the TMA form, the work items' meta bits, the alignment of
the tensor maps in the job descriptors and the persistent kernels' shared-memory requests."""
import os
import subprocess

import pytest

from paper_2509_12494_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2509_12494_gb300", "csrc")


def test_host_tables(tmp_path):
    try:
        nvcc = _build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "host_tables_check")
    r = subprocess.run([nvcc, *_build.ARCH, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC,
                        os.path.join(ROOT, "tests", "host_tables_check.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-4000:]
