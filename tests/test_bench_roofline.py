"""bench.py's roofline helpers on the CPU: the recorded DRAM traffic of a kernel
is reported only for the kernel sources it was captured on, the FP32 peak comes
from the unit counts and the sampled clock, the HBM peak from the measured-peaks
file (else the stated fallback)."""
import hashlib
import json
import os

import pytest

import bench


def _source_hash():
    h = hashlib.sha256()
    for name in ("dslash.cu", "common.cuh"):
        with open(os.path.join(bench.ROOT, "paper_1104_0737_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def test_traffic_only_for_the_captured_source(monkeypatch):
    records = {("k", "w"): {"bytes": 123, "source_sha256": _source_hash()},
               ("k", "old"): {"bytes": 456, "source_sha256": "0" * 16}}
    monkeypatch.setattr(bench, "NCU_TRAFFIC", records)
    assert bench.ncu_traffic("k", "w") == 123
    assert bench.ncu_traffic("k", "old") is None  # the kernel changed since the capture
    assert bench.ncu_traffic("k", "unrecorded") is None


def test_recorded_traffic_is_near_the_algorithmic_bytes():
    """Each record is one launch at 32^3 x 64, L = 12: its DRAM bytes lie within
    a few tens of percent of the algorithmic bytes (a record of the wrong kernel
    or workload would not)."""
    V, L = 32 ** 3 * 64, 12
    alg = {"sap_sweep": bench.sap_sweep_bytes(V, L),
           "sap_resid": bench.sap_resid_bytes(V, L, (8, 8, 8, 8), link_reals=bench.FP32_LINK_REALS)}
    for (kernel, workload), rec in bench.NCU_TRAFFIC.items():
        assert workload == "wilson_32c64_L12"
        assert 0.8 < rec["bytes"] / alg[kernel] < 1.25, kernel


def test_fp32_peak_from_unit_counts():
    assert bench.fp32_alu_peak_tflops(2070) == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)


def test_hbm_peak_from_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6786.6}))
    assert bench.load_peaks() == (6786.6, "measured")
