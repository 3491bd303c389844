"""The bench line's host-side assembly (no GPU): the compact summary is the line's last key, stays
short enough to survive a kept tail of the line, and carries every configuration's headline."""
import json
import sys

import pytest


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    import bench as B
    return B


def _fake_line():
    pts = [{"mode": m, "load": f, "of": o, "p50_ms": 0.7512, "p99_ms": 1.512, "jobs_per_s": 123456.7}
           for m, f, o in (("batched", 0.5, "batched"), ("batched", 1.0, "batched"), ("batched", 1.25, "batched"),
                           ("plain", 0.5, "plain"), ("plain", 1.0, "plain"), ("plain", 0.5, "batched"))]
    return {"metric": "m", "value": 1.0, "ms_per_step": 1.4181, "config": {"q_bits": 124},
            "roundtrip_bit_exact": True, "forward_sampled_bit_exact": True,
            "batched_call": {"ms_per_step": 1.384}, "plain": {"ms_per_step": 6.3},
            "e2e": {"ms_per_step": 1.65}, "roofline": {"frac": 0.583},
            "c3_other_width": {"q_bits": 60, "ms_batched": 0.72, "ms_call": 0.70, "ms_plain": 5.4,
                               "roundtrip_bit_exact": True, "forward_sampled_bit_exact": True},
            "uneven": {"ms_per_step": 5.06, "per_call": {"ms_per_step": 19.6}, "modmul_per_s": 1.72e11,
                       "jobs_bit_exact_vs_per_call": True, "forward_jobs_bit_exact_vs_per_call": True,
                       "autotuned": {"form": "prefetch", "ctas_per_sm": 3, "lag": 4, "blas_chunk": 16384,
                                     "split_shift": -1, "tune_s": 4.2}},
            "serve": {"saturated_jobs_per_s": {"batched": 1.82e5, "plain": 1.98e4}, "points": pts},
            "blas": {k: {"GB/s": 6000.0} for k in ("vadd_124", "vmul_124", "axpy_124", "vadd_60", "vmul_60")},
            "small_ntt": {"calls_us": 17.9, "graph_us": 22.8, "roundtrip_bit_exact": True},
            "cpu_baseline": {"value": 2.9e6}}


def test_summary_is_last_and_short(bench):
    out = bench.tail_summary(_fake_line())
    assert list(out)[-1] == "summary"
    line = json.dumps(out)
    tail = line[line.index('"summary"'):]
    assert len(tail) < 1300, len(tail)
    s = out["summary"]
    assert s["c3"]["ms_call"] == 1.384 and s["c3"]["fwd_exact"] is True
    assert s["c3_other"]["bits"] == 60 and s["c4"]["exact"] is True and s["c4"]["tuned"]["lag"] == 4
    assert "tune_s" not in s["c4"]["tuned"]
    assert len(s["c5"]["p50_p99_ms_jobs_per_s"]) == 6 and s["c1_us"]["graph"] == 22.8


def test_summary_tolerates_missing_blocks(bench):
    line = _fake_line()
    for k in ("c3_other_width", "uneven", "serve", "blas", "small_ntt", "plain"):
        line.pop(k)
    s = bench.tail_summary(line)["summary"]
    assert set(s) == {"c3"} and s["c3"]["ms_plain"] is None


def test_algorithmic_counts_follow_the_scope_table(bench):
    # 30 limb products of a 124-bit Shoup product, two instructions each; 36 for Barrett
    assert bench.MADS_PER_SHOUP == {1: 16, 2: 60} and bench.MADS_PER_BARRETT[2] == 72
    assert bench.brv(1, 16) == 1 << 15 and bench.residue_int([1, 2], 2) == 1 + (2 << 64)
