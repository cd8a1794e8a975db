"""Host logic of bench.py that decides what its JSON line reports, checked on the CPU.

- The clock summary: the median SM clock under load, and the throttle reasons seen active
  in nvidia-smi's samples. A run that saw a thermal or hardware slowdown is rejected, so
  these must be read right.
- The committed DRAM-traffic constant: it is reported only for the kernel sources it was
  captured on and only at the tile size it was captured at, and it is scaled by the launch's
  keys. Otherwise the line carries null.
- The garbage collector is held off inside a timed region and restored after it.
"""
import gc
import json
import shutil

import pytest

import bench

HDR_SAMPLE = "0, {sm}, 2032, 800.5, {act}, {hw}, {hwt}, {swt}, {swp}"


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s


def test_clock_summary_median_and_reasons():
    ok = "Not Active"
    lines = [HDR_SAMPLE.format(sm=m, act="0x0", hw=ok, hwt=ok, swt=ok, swp=ok) for m in (2032, 2017, 2032)]
    lines.append(HDR_SAMPLE.format(sm=1950, act="0x4", hw=ok, hwt=ok, swt=ok, swp="Active"))
    lines.append("garbage line")
    lines.append("0, [N/A], 2032, 1, 0x0, a, b, c, d")   # unparsable clock: skipped
    d = _sampler(lines).summary()
    assert d["samples"] == 4 and d["sm_max_mhz"] == 2032.0
    assert d["sm_mhz"] == pytest.approx(2024.5)
    assert d["reasons"] == ["sw_power_cap"]
    hot = HDR_SAMPLE.format(sm=1500, act="0x40", hw=ok, hwt="Active", swt="Active", swp=ok)
    assert _sampler([hot]).summary()["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    empty = _sampler([]).summary()
    assert empty["samples"] == 0 and empty["reasons"] == ["unavailable"]


def _fake_root(tmp_path, entry, sources_text):
    """A repository root holding one traffic constant and the kernel sources it names."""
    root = tmp_path / "root"
    csrc = root / "paper_2512_08478_b300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in sources_text.items():
        (csrc / name).write_text(text)
    (root / "profiles").mkdir()
    (root / "profiles" / "traffic.json").write_text(json.dumps({"composite": entry}))
    return root


def test_committed_traffic_is_keyed_by_sources_and_tile(tmp_path, monkeypatch):
    srcs = {"composite.cu": "kernel v1\n", "splat_eval.cuh": "helpers\n"}
    entry = dict(bytes_per_key=22.5, sources=list(srcs), tile=32)
    root = _fake_root(tmp_path, entry, srcs)
    monkeypatch.setattr(bench, "ROOT", root)
    entry["source_sha"] = bench._kernel_sha(entry["sources"])
    (root / "profiles" / "traffic.json").write_text(json.dumps({"composite": entry}))
    assert bench._committed_traffic("composite", 1_000_000, 5, tile=32) == 22_500_000
    assert bench._committed_traffic("composite", 1_000_000, 5, tile=16) is None   # another tile size
    assert bench._committed_traffic("preprocess", 1_000_000, 5) is None           # no constant
    (root / "paper_2512_08478_b300" / "csrc" / "composite.cu").write_text("kernel v2\n")
    assert bench._committed_traffic("composite", 1_000_000, 5, tile=32) is None   # kernel changed
    shutil.rmtree(root / "profiles")
    assert bench._committed_traffic("composite", 1_000_000, 5, tile=32) is None   # no file


def test_committed_traffic_per_gaussian_without_tile(tmp_path, monkeypatch):
    srcs = {"preprocess.cu": "k\n"}
    root = _fake_root(tmp_path, {}, srcs)
    monkeypatch.setattr(bench, "ROOT", root)
    entry = dict(bytes_per_gaussian=285.5, sources=list(srcs), source_sha=bench._kernel_sha(list(srcs)))
    (root / "profiles" / "traffic.json").write_text(json.dumps({"preprocess": entry}))
    assert bench._committed_traffic("preprocess", 7, 2_000_000, tile=16) == 571_000_000


def test_clock_sampler_holds_the_collector_off(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: (_ for _ in ()).throw(OSError("no smi")))
    was = gc.isenabled()
    gc.enable()
    try:
        with bench.ClockSampler(0):
            assert not gc.isenabled()
        assert gc.isenabled()
        gc.disable()
        with bench.ClockSampler(0):
            assert not gc.isenabled()
        assert not gc.isenabled()   # a collector that was off stays off
    finally:
        (gc.enable if was else gc.disable)()
