"""Host-side arithmetic of bench.py (no GPU): the algorithmic work per stage
launch, the whole-job value, and the ncu traffic entry, which is scaled from its
capture by the spectrum size and withheld once the stage kernels' sources
differ from the ones captured."""

import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_at_5000x10000():
    b = bench.algorithmic_bytes(5000, 10000)
    spec = 16 * 5000 * 5002                     # [n_theta][Kp] complex doubles, Kp = 5002
    grid = 8 * 5000 * 10000                     # f or u
    assert b["theta_inverse"] == b["theta_forward"] == 2 * spec == 800_320_000
    assert b["rows_forward"] == b["rows_inverse"] == grid + spec
    assert b["solve"] == 2 * spec + 3 * 8 * 5000 * 5002
    # FP32 spectrum and tables
    b32 = bench.algorithmic_bytes(5000, 10000, spec_elem=8, table_elem=4)
    assert b32["theta_forward"] == 2 * 8 * 5000 * 5002
    # fused: the spectrum in and out once, one FP32 pivot per (j, k) of the 5001 columns
    assert b32["theta_fused"] == 2 * 8 * 5000 * 5002 + 4 * 5000 * 5001


def test_algorithmic_flops_are_the_conventional_counts():
    f = bench.algorithmic_flops(5000, 10000)
    assert f["rows_forward"] == pytest.approx(5000 * 2.5 * 10000 * math.log2(10000))
    assert f["theta_forward"] == pytest.approx(5001 * 5.0 * 5000 * math.log2(5000))
    assert f["solve"] == 10.0 * 5000 * 5001
    stages = ("rows_forward", "theta_forward", "solve", "theta_inverse", "rows_inverse")
    per_dof = sum(f[s] for s in stages) / (5000 * 10000)
    assert 130 < per_dof < 145                  # ~5 log2(n N) + 10
    # the fused colatitude stage of the FP32 form does both transforms and the solve
    assert f["theta_fused"] == pytest.approx(f["theta_forward"] + f["solve"] + f["theta_inverse"])


def test_whole_job_value_counts_every_rank():
    assert bench.whole_job_value(50_000_000, 1, 10.0) == pytest.approx(5e9)
    assert bench.whole_job_value(50_000_000, 4, 10.0) == pytest.approx(2e10)


def test_traffic_is_scaled_from_the_capture_and_withheld_on_changed_sources(monkeypatch):
    cap = bench.TRAFFIC_CAPTURE
    cap32 = bench.TRAFFIC_CAPTURE_FP32
    monkeypatch.setattr(bench, "csrc_hash",
                        lambda sources=bench.TRAFFIC_SOURCES: cap32["csrc_sha256"] if "fused.cuh" in sources
                        else cap["csrc_sha256"])
    t, note = bench.traffic_for("theta_inverse", cap["n_theta"], cap["n_lambda"], "fp64")
    assert t == cap["bytes"]["theta_inverse"]
    t2, _ = bench.traffic_for("theta_inverse", 5000, 10000, "fp64")
    assert t2 == int(cap["bytes"]["theta_inverse"] * (5000 * 5002) / (5000 * 2502))
    # the FP32 form has a capture of its fused colatitude stage only
    assert bench.traffic_for("theta_inverse", 5000, 10000, "fp32")[0] is None
    t32, _ = bench.traffic_for("theta_fused", 5000, 10000, "fp32")
    assert t32 == int(cap32["bytes"]["theta_fused"] * (5000 * 5002) / (5000 * 2502))
    assert bench.traffic_for("theta_fused", 5000, 10000, "fp32_refine")[0] is None
    monkeypatch.setattr(bench, "csrc_hash", lambda sources=bench.TRAFFIC_SOURCES: "0" * 16)
    t3, why = bench.traffic_for("theta_inverse", 5000, 10000, "fp64")
    assert t3 is None and "changed" in why


def test_source_hash_covers_the_stage_kernel_sources():
    h = bench.csrc_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    for name in bench.TRAFFIC_SOURCES + bench.TRAFFIC_SOURCES_FP32:
        assert os.path.exists(os.path.join(ROOT, "paper_1510_08094_gb300", "csrc", name))
