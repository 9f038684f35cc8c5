"""Host logic of bench.py that the reported numbers rest on, without a GPU:
the algorithmic byte model of the product, the DRAM-traffic lookup and its
staleness rule, the clock-sample summary and the peak lookup."""
import os
import types

import pytest

import bench


def _fake_handle(shape, lengths, n_panels):
    return types.SimpleNamespace(shape=shape, N=n_panels, fft_lengths=lambda: lengths)


def test_model_bytes_by_hand():
    # 4x6x2 grid padded to 10x14x6: Hx = 6, octant 6*8*4, z-unpadded planes Nz+1 = 3
    vc = _fake_handle((4, 6, 2), (10, 14, 6), 100)
    spectra = 15 * 4 * 6 * 8 * 4
    inter = 2 * 9 * 8 * 6 * 14 * 3
    assert bench.mvm_model_bytes(vc, 1) == 12 * 100 + spectra + inter
    # the spectra are read once per batched product, shared by its columns
    assert bench.mvm_model_bytes(vc, 4) == 12 * 100 + spectra / 4 + inter


def test_traffic_follows_the_source_digest(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "product_sources_hash", lambda: "0123456789abcdef")
    assert bench.captured_traffic("bus") is None                 # no capture at all
    (prof / "product_traffic_bus.md").write_text(
        "# capture\n\ntraffic_bytes_per_product: 4441414400 sources: 0123456789abcdef\n")
    assert bench.captured_traffic("bus") == 4441414400
    monkeypatch.setattr(bench, "product_sources_hash", lambda: "fedcba9876543210")
    assert bench.captured_traffic("bus") is None                 # kernels changed since
    (prof / "product_traffic_bus.md").write_text("# capture without a digest line\n")
    assert bench.captured_traffic("bus") is None


def test_source_digest_covers_every_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2004_02609_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in ("a.cu", "b.cuh", "c.h"):
        (csrc / name).write_text("// " + name + "\n")
    (csrc / "notes.txt").write_text("not a source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.product_sources_hash()
    assert d0 == bench.product_sources_hash()
    (csrc / "notes.txt").write_text("changed\n")
    assert bench.product_sources_hash() == d0
    for name in ("a.cu", "b.cuh", "c.h"):
        before = bench.product_sources_hash()
        (csrc / name).write_text("// " + name + " edited\n")
        assert bench.product_sources_hash() != before


def test_committed_captures_name_their_digest():
    for wl in ("meanders", "bus"):
        p = os.path.join(bench.ROOT, "profiles", f"product_traffic_{wl}.md")
        txt = open(p).read()
        assert "traffic_bytes_per_product:" in txt and "sources:" in txt
        assert "--clock-control none" in txt


def test_clock_summary(tmp_path):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    open(s.path, "w").write("\n".join(rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not os.path.exists(s.path)
    s.path = str(tmp_path / "missing.csv")
    assert s.summary()["reasons"] == ["unsampled"]


def test_peak_lookup(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6780.5}')
    assert bench.read_peaks() == (6780.5, "measured")


@pytest.mark.parametrize("name", ["plates", "bus", "pillars", "meanders", "meanders256"])
def test_workloads_are_described(name):
    w, desc = bench.workload(name)
    assert w.labels.ndim == 3 and len(desc) > 10
