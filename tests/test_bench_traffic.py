"""bench.py's roofline.traffic comes from the committed ncu summary only while
the kernel's source is byte for byte the one the counters were taken on."""
import hashlib
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sha(names):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2004_11040_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def test_committed_traffic_matches_the_sources():
    """Both hot kernels have counters for their current sources, per lifting of
    the bench step (10 legs at N = 2^20, k = 1024), between the algorithmic
    bytes and a few times them."""
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for kernel in ("k_run", "k_run_graph"):
        k = d["kernels"][kernel]
        if k["sources_sha256"] != _sha(k["sources"]):
            # a source edited since the capture: bench.py reports traffic as null
            assert b.traffic_for(kernel) is None
            pytest.skip(f"{kernel}: source changed since the ncu capture")
        per = b.traffic_for(kernel)
        assert per == k["dram_bytes_per_launch"] / k["liftings_in_captured_launch"]
        assert per == k["dram_bytes_per_lifting"]
        assert 0.5 * b.BYTES_PER_LIFTING <= per < 4 * b.BYTES_PER_LIFTING, (kernel, per)


def test_traffic_is_null_once_a_source_changes(tmp_path, monkeypatch):
    b = _bench()
    prof = tmp_path / "profiles"
    csrc = tmp_path / "paper_2004_11040_gb300" / "csrc"
    prof.mkdir()
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(b"kernel A")
    (csrc / "k.cuh").write_bytes(b"header A")
    h = hashlib.sha256(b"kernel A" + b"header A").hexdigest()
    entry = {"sources": ["k.cu", "k.cuh"], "sources_sha256": h, "dram_bytes_per_lifting": 123.5}
    (prof / "traffic.json").write_text(json.dumps({"kernels": {"k_x": entry}}))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.traffic_for("k_x") == 123.5
    (csrc / "k.cuh").write_bytes(b"header B")
    assert b.traffic_for("k_x") is None
    assert b.traffic_for("k_missing") is None
