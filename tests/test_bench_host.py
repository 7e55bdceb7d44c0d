"""The bench's host-side arithmetic on CPU: the per-kernel rooflines, the scaling of the
committed ncu traffic table to a launch, the stratified trace samples and the throughput
aggregation."""
import json
import os

import numpy as np
import pytest

import bench


def test_roofline_takes_the_longer_replay_kernel_with_its_own_bytes():
    # k_phase1 reads 17 B per first-unit event and 8 B per sketched event; k_final 17 B per
    # event of the other units; k_copy 13 B per memcpy
    n, m, first = 1_000_000, 100_000, 400_000
    kt = {"phase1": (8.0, 2), "final": (3.0, 2), "copy": (0.6, 2), "compact": (1.0, 2), "reset": (0.5, 2)}
    r = bench.roofline_of(kt, n=n, m=m, first_events=first, traffic=False)
    assert r["kernel"] == "phase1"
    alg = 17.0 * first + 8.0 * (n - first)
    assert r["alg_bytes"] == pytest.approx(alg)
    assert r["achieved"] == pytest.approx(alg / (4.0 / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["kernels"]["final"]["achieved"] == pytest.approx(17.0 * (n - first) / (1.5 / 1e3) / 1e9)
    assert r["kernels"]["copy"]["achieved"] == pytest.approx(13.0 * m / (0.3 / 1e3) / 1e9)
    assert r["traffic"] is None


def test_traffic_table_matches_the_kernel_sources_or_is_withheld(monkeypatch):
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        assert bench.traffic_for("phase1", 1000.0) is None
        return
    d = json.load(open(path))
    k = d["kernels"]
    for name in ("phase1", "final", "copy"):
        assert k[name]["dram_bytes_per_streamed_byte"] == pytest.approx(k[name]["dram_bytes"] / k[name]["streamed_bytes"])
    # the captured case's streamed bytes follow from its event counts
    c = d["case"]
    sb = bench.streamed_bytes(c["events"], c["memcpys"], c["first_events"], c["sketch_events"])
    for name in ("phase1", "final", "copy"):
        assert k[name]["streamed_bytes"] == pytest.approx(sb[name])
    if k["final"]["source_hash"] == bench.source_hash("final"):
        assert bench.traffic_for("final", 1000.0) == pytest.approx(k["final"]["dram_bytes_per_streamed_byte"] * 1000.0)
    # a changed kernel source withholds the figure
    monkeypatch.setattr(bench, "source_hash", lambda kernel: "0" * 16)
    assert bench.traffic_for("final", 1000.0) is None


def test_batched_sample_spans_the_lengths_and_keeps_every_leaking_trace():
    lens, mlen = bench.batched_spec(4096)
    pick = bench.batched_sample(lens)
    assert int(np.argmin(lens)) in pick and int(np.argmax(lens)) in pick
    assert all(i in pick for i in range(0, 4096, 100))
    assert 512 <= len(pick) <= 512 + 41
    # the sample's length distribution follows the batch's (evenly spaced ranks)
    assert abs(np.median(lens[pick]) / np.median(lens) - 1) < 0.05
    sub = bench.parity_subset(lens, pick)
    assert int(np.argmin(lens)) in sub and int(np.argmax(lens)) in sub
    assert all(i in sub for i in range(0, 4096, 100))


def test_reference_and_gpu_arms_name_the_same_configuration():
    lens, mlen = bench.batched_spec(4096)
    a = bench.batched_config(4096, lens, mlen)
    b = bench.batched_config(4096, *bench.batched_spec(4096))
    assert a == b and a["memcpys"] == int(mlen.sum()) and a["n_lines"] == 4096


def test_aggregate_is_all_events_over_the_slowest_rank():
    v, t = bench.aggregate([10.0, 20.0], [1000, 3000])
    assert t == 20.0 and v == pytest.approx(4000 / 0.020)


def test_default_workload_is_the_batched_configuration():
    assert bench.parse([]).workload == "batched"


def test_stride_case_keeps_the_batch_length_mix():
    ids = bench.batched_ids(256, 16)
    assert list(ids[:3]) == [0, 16, 32] and len(ids) == 256
    lens, mlen = bench.batched_spec(256, 0, 0, 16)
    full, _ = bench.batched_spec(4096)
    assert np.array_equal(lens, full[ids]) and np.array_equal(mlen, lens // 10)
    assert "every 16th" in bench.batched_config(256, lens, mlen, 16)["workload"]


def test_streamed_bytes_add_the_sketch_warmups_to_phase1_only():
    n, m, first = 10_000_000, 1_000_000, 4_000_000
    alg = bench.kernel_bytes(n, m, first)
    sb = bench.streamed_bytes(n, m, first, sketch_streamed=6_500_000)
    assert sb["final"] == alg["final"] and sb["copy"] == alg["copy"]
    assert sb["phase1"] - alg["phase1"] == pytest.approx(8.0 * (6_500_000 - (n - first)))
    assert bench.streamed_bytes(n, m, first) == alg


def test_each_kernel_hashes_its_own_sources():
    h = {k: bench.source_hash(k) for k in bench.KERNEL_SOURCES}
    assert len(set(h.values())) == 3 and all(len(v) == 16 for v in h.values())
    assert all("scl_post.cu" not in files for files in bench.KERNEL_SOURCES.values())
