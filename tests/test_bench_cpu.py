"""CPU checks of bench.py's host logic for the roofline's `traffic` key: the
ncu DRAM-traffic record is used only while the sources it lists are byte for
byte those it was captured from, and it is scaled to a launch by algorithmic
bytes.  No GPU is touched."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record(tmp_path, files, dram=970, alg=1000):
    h = hashlib.sha256()
    for f in files:
        h.update((tmp_path / f).read_bytes())
    rec = {"mg_fwd": {"dram_bytes_per_launch": dram, "algorithmic_bytes_per_launch": alg,
                      "sources": list(files), "source_sha256": h.hexdigest()}}
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))


def test_traffic_record_is_scaled_and_voided_by_a_source_change(tmp_path, monkeypatch):
    (tmp_path / "a.cu").write_text("kernel, first version")
    (tmp_path / "b.cuh").write_text("header")
    _record(tmp_path, ["a.cu", "b.cuh"])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # 970 DRAM bytes for 1000 algorithmic bytes, scaled to a launch of 500
    assert bench.read_traffic("mg_fwd", 500) == pytest.approx(485.0)
    assert bench.read_traffic("mg_y", 500) is None
    (tmp_path / "b.cuh").write_text("header, edited")
    assert bench.read_traffic("mg_fwd", 500) is None
    (tmp_path / "b.cuh").write_text("header")
    assert bench.read_traffic("mg_fwd", 500) == pytest.approx(485.0)
    (tmp_path / "a.cu").unlink()
    assert bench.read_traffic("mg_fwd", 500) is None


def test_traffic_record_without_file_is_none(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic("mg_fwd", 500) is None


def test_committed_traffic_record_is_well_formed():
    """The committed record names sources that exist, and its algorithmic
    bytes are the kernel's own count for the captured launch: 160 slices of
    512^2, 6.25 FP32 maps per pixel (z, p, r, a^2 in; z, r out; a quarter map
    of level-1 residual out; q = M p is formed again from p)."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["mg_fwd"]
    assert rec["sources"] and all(os.path.isfile(os.path.join(ROOT, s)) for s in rec["sources"])
    assert "paper_2308_01290_gb300/csrc/solver.cu" in rec["sources"]
    assert rec["algorithmic_bytes_per_launch"] == 160 * 512 * 512 * 4 * 25 // 4
    assert rec["dram_bytes_per_launch"] == rec["dram_read"] + rec["dram_write"]
    assert 0.5 < rec["dram_bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] < 1.5


def test_fifo_latencies_of_one_server():
    """The one-at-a-time baseline of the serving leg: a request starts when it
    arrives or when the previous one finishes, whichever is later."""
    import bench
    arr = np.array([0.0, 0.5, 0.6, 5.0])
    svc = np.array([1.0, 1.0, 0.2, 0.5])
    lat, end = bench.fifo_latencies(arr, svc)
    # finishes: 1.0, 2.0, 2.2, 5.5
    assert np.allclose(lat, [1.0, 1.5, 1.6, 0.5]) and end == 5.5
    # Poisson arrival times are seeded and increasing
    a = bench.poisson_arrivals(50.0, 200, 3)
    assert np.all(np.diff(a) > 0) and np.array_equal(a, bench.poisson_arrivals(50.0, 200, 3))
    assert 2.0 < a[-1] < 6.0
