"""Host logic of bench.py that needs no GPU: the ncu traffic record is reported
only while the kernel sources hash to the value it was captured on."""
import json
import os

import bench


def _record(tmp_path, h):
    os.makedirs(tmp_path / "profiles", exist_ok=True)
    rec = {"tgv256:fp32": {"kernel_hash": h, "dram_bytes_per_step": 123.0}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))


def test_traffic_reported_only_for_the_captured_kernel_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "abc")
    assert bench.profile_traffic("tgv256:fp32") is None             # no record
    _record(tmp_path, "abc")
    assert bench.profile_traffic("tgv256:fp32") == 123.0
    assert bench.profile_traffic("tgv256:fp64") is None             # another workload
    _record(tmp_path, "stale")
    assert bench.profile_traffic("tgv256:fp32") is None             # kernels changed since


def test_kernel_hash_covers_the_step_sources():
    h0 = bench.kernel_hash()
    assert len(h0) == 16 and h0 == bench.kernel_hash()
    assert "lbm_fused.cuh" in bench.KERNEL_SOURCES and "lbm_ops.cuh" in bench.KERNEL_SOURCES
