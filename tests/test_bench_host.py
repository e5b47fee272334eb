"""Host-side pieces of bench.py that need no GPU: the committed DRAM-traffic
profile is used only for the interior-kernel sources it was captured at,
and the clock sampler degrades to a line without samples where neither NVML
nor nvidia-smi is there."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    import bench as b

    return b


def _write_profile(tmp_path, top_hash, formats):
    d = tmp_path / "profiles"
    d.mkdir()
    (d / "interior_step_traffic.json").write_text(json.dumps({"source_hash": top_hash, "formats": formats}))
    return str(tmp_path)


def test_traffic_is_read_only_at_the_sources_it_was_captured_at(bench, tmp_path, monkeypatch):
    here = bench.kernel_source_hash()
    root = _write_profile(tmp_path, here, {
        "f32h": {"dram_bytes_per_node": 106.4},
        "f32c": {"dram_bytes_per_node": 114.6, "source_hash": "0000000000000000"},
    })
    monkeypatch.setattr(bench, "ROOT", root)
    # the hash is of the kernel's sources, which stay where they are
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: here)
    assert bench.ncu_traffic("f32", "lo16", 1000) == pytest.approx(106400.0)
    # a format captured at other sources, and one never captured: no figure
    assert bench.ncu_traffic("f32", "pair", 1000) is None
    assert bench.ncu_traffic("bf16", "pair", 1000) is None


def test_traffic_at_other_sources_is_not_used(bench, tmp_path, monkeypatch):
    here = bench.kernel_source_hash()
    root = _write_profile(tmp_path, "ffffffffffffffff", {"f32h": {"dram_bytes_per_node": 106.4}})
    monkeypatch.setattr(bench, "ROOT", root)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: here)
    assert bench.ncu_traffic("f32", "lo16", 1000) is None


def test_committed_traffic_profile_names_its_sources(bench):
    with open(os.path.join(ROOT, "profiles", "interior_step_traffic.json")) as fh:
        d = json.load(fh)
    assert len(d["source_hash"]) == 16 and "command" in d
    for key, e in d["formats"].items():
        assert e["dram_bytes_per_node"] > 0, key


def _nvml_loads():
    import ctypes

    try:
        ctypes.CDLL("libnvidia-ml.so.1")
        return True
    except OSError:
        return False


@pytest.mark.skipif(_nvml_loads(), reason="the driver's NVML library is present: the sampler would read a GPU")
def test_clock_sampler_without_a_gpu_returns_no_samples(bench, monkeypatch):
    monkeypatch.setenv("PATH", "/nonexistent")
    s = bench.clock_sampler(0)
    s.start()
    assert s.stop() is None
