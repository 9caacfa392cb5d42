"""Host logic of bench.py that needs no GPU: the ncu traffic record is reported
only while the library sources hash to the value it was captured on, and the
CPU leg times the oracle on one core and on every host core."""
import json
import os
import shutil

import numpy as np

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


def test_kernel_hash_covers_every_library_source(tmp_path, monkeypatch):
    """Editing any file under csrc/ or include/, or the build script, changes the hash."""
    root = bench.ROOT
    shutil.copytree(os.path.join(root, "paper_2510_14712_gb300", "csrc"),
                    tmp_path / "paper_2510_14712_gb300" / "csrc")
    shutil.copytree(os.path.join(root, "include"), tmp_path / "include")
    shutil.copy(os.path.join(root, "paper_2510_14712_gb300", "build.py"), tmp_path / "paper_2510_14712_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    assert len(h0) == 16 and h0 == bench.kernel_hash()
    files = bench.kernel_sources()
    names = {os.path.basename(f) for f in files}
    for f in os.listdir(os.path.join(root, "paper_2510_14712_gb300", "csrc")):
        assert f in names, f
    assert "build.py" in names and "lbm.h" in names
    for f in files:
        data = open(f, "rb").read()
        with open(f, "ab") as fh:
            fh.write(b" ")
        assert bench.kernel_hash() != h0, f
        with open(f, "wb") as fh:
            fh.write(data)
    assert bench.kernel_hash() == h0


def test_cpu_leg_one_core_and_all_cores(tmp_path):
    """The oracle is timed on one core (saving its final fields) and then on every
    host core at once, one process each; the saved step count includes the warm-up."""
    path = str(tmp_path / "ref.npz")
    r = bench.cpu_oracle_leg("riemann", steps=2, warmup=1, save=path)
    assert "error" not in r and "all_cores_error" not in r, r
    assert r["cores"] == bench.host_cores()
    assert r["value"] > 0 and r["single_core"]["value"] > 0 and r["model"]
    assert "processes" in r["sample"] and r["kind"] == "oracle"
    ref = np.load(path)
    assert int(ref["steps"]) == 3 and ref["rho"].shape == (4, 1000) and ref["u"].shape == (2, 4, 1000)
