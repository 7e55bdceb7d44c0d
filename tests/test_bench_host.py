"""The bench's host-side arithmetic on CPU: the dominant-kernel roofline and the scaling of
the committed ncu traffic table to a launch."""
import json
import os

import pytest

import bench


def test_roofline_takes_an_event_path_kernel_and_its_own_units():
    # the copy kernel's span is the longest (it waits beside the event path) but is not chosen
    kt = {"sketch": (8.0, 10), "final": (9.0, 10), "copy_apply": (20.0, 10), "scan": (1.0, 10)}
    r = bench.roofline_of(kt, n=1_000_000, m=100_000, traffic=False, sketch_n=900_000)
    assert r["kernel"] == "final"
    # 17 B per event over the events the exact replay takes (first units excluded), per launch
    assert r["achieved"] == pytest.approx(17.0 * 900_000 / (0.9 / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None


def test_traffic_table_matches_the_kernel_sources_or_is_withheld(tmp_path, monkeypatch):
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    k = d["kernels"]
    for name, unit in (("sketch", "streamed event"), ("final", "event"), ("copy_apply", "memcpy")):
        assert k[name]["unit"] == unit
    # the table is read only when its hash is the current sources'
    if d["source_hash"] == bench.source_hash():
        assert bench.traffic_for("sketch", 10, streamed=1000) == pytest.approx(k["sketch"]["dram_bytes_per_unit"] * 1000)
        assert bench.traffic_for("final", 1000) == pytest.approx(k["final"]["dram_bytes_per_unit"] * 1000)
    # a changed kernel source withholds the figure
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.traffic_for("final", 1000) is None


def test_measured_traffic_is_close_to_the_algorithmic_bytes():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["kernels"]
    assert d["sketch"]["dram_bytes_per_unit"] == pytest.approx(bench.ALG_BYTES["sketch"], rel=0.05)
    assert d["final"]["dram_bytes_per_unit"] == pytest.approx(bench.ALG_BYTES["final"], rel=0.05)
    assert d["copy_apply"]["dram_bytes_per_unit"] == pytest.approx(bench.ALG_BYTES["copy_apply"], rel=0.05)


def test_aggregate_is_all_events_over_the_slowest_rank():
    v, t = bench.aggregate([10.0, 20.0], [1000, 3000])
    assert t == 20.0 and v == pytest.approx(4000 / 0.020)
