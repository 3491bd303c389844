"""Host-side behaviour that needs no GPU: the binding refuses to run without the CUDA library, and
the benchmark's reference arm (the oracle on the host cores) prints a complete JSON line."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_2509_12494_gb300 import _build
    from paper_2509_12494_gb300 import mqntt as M
    monkeypatch.setattr(M, "_lib", None)
    monkeypatch.setattr(_build, "LIB", os.path.join(ROOT, "no-such-dir", "libmqntt.so"))
    with pytest.raises(RuntimeError, match="missing"):
        M.load()


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--batch", "16", "--log2n", "10"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "butterflies/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["batch"] == 16 and line["config"]["log2n"] == 10
