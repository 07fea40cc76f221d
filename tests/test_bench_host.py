"""bench.py's host-side logic on the CPU (no GPU): the roofline's byte model,
the DRAM-traffic figure and its link to the committed ncu capture, the
serving workloads' sizes, and the comparison of served results with the jobs
run alone."""
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILE = os.path.join(ROOT, "profiles", "layer_kernel_ring32_zn_layer19.md")


def test_byte_model():
    # 16 B key per update of a scanned gate; 64 B per anticommuting term
    assert bench.BYTES_PER_ANTICOMMUTING == 64
    assert bench.algorithmic_bytes(100, 0, 0) == 1600
    assert bench.algorithmic_bytes(100, 40, 0) == 960
    assert bench.algorithmic_bytes(100, 40, 10) == 960 + 640


def test_traffic_capture_is_the_committed_profile():
    """The ratio and digest bench.py scales traffic with are those of the
    committed capture: DRAM bytes over algorithmic bytes of the same launch,
    kernel sources with the same digest."""
    text = open(PROFILE).read()
    assert "digest " + bench.TRAFFIC_CAPTURE["sources_sha16"] in text
    dram = float(re.search(r"= ([\d.]+) GB \(([\d.]+) x algorithmic\)", text).group(1))
    alg = float(re.search(r"\| algorithmic bytes [^|]*\| ([\d.]+) GB \|", text).group(1))
    assert bench.TRAFFIC_CAPTURE["ratio"] == pytest.approx(dram / alg, rel=2e-3)


def test_traffic_is_null_when_the_kernel_sources_change(monkeypatch):
    here = bench.kernel_sources_sha16()
    assert re.fullmatch(r"[0-9a-f]{16}", here)
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "sources_sha16", here)
    assert bench.traffic_per_launch(1e9) == pytest.approx(bench.TRAFFIC_CAPTURE["ratio"] * 1e9)
    monkeypatch.setitem(bench.TRAFFIC_CAPTURE, "sources_sha16", "0" * 16)
    assert bench.traffic_per_launch(1e9) is None


def test_scaled_serving_stream_sizes():
    specs = bench.serving_specs(300, 200.0)
    assert len(specs) == 300
    arrivals = [a for a, _ in specs]
    assert arrivals == sorted(arrivals) and 0.5 < arrivals[-1] < 3.0  # ~1.5 s of arrivals
    for _, wl in specs:
        n, steps = wl.circuit.n, len(wl.circuit.layers)
        assert wl.eps >= 1e-4
        if wl.noise_mode == 0 and n in (16, 32, 64, 128) and wl.max_weight == 8:
            assert steps <= 20  # ring
        else:
            assert n in (8, 10, 12, 16) and steps <= 4  # all-to-all Heisenberg


def test_full_serving_stream_prefix_sizes():
    specs = bench.serving_specs_full(40, 200.0)
    assert len(specs) == 40
    for _, wl in specs:
        assert wl.circuit.n in (16, 32, 64, 128)
        assert 1e-6 <= wl.eps <= 1e-3
        steps = len(wl.circuit.layers)
        assert 5 <= steps <= 40
        if wl.noise_mode == 1:  # all-to-all with per-gate damping
            assert wl.noise_p == 0.01 and wl.symmetry in (0, 2)
        else:  # ring, weight <= 10
            assert wl.max_weight == 10 and wl.symmetry in (0, 1)


def test_served_results_against_alone():
    res = [{"status": 0, "value": 0.5}, {"status": 0, "value": 0.25}, {"status": 3, "value": 9.0}]
    alone = [{"status": 0, "value": 0.5 + 2.0 ** -52}, {"status": 0, "value": 0.25},
             {"status": 0, "value": 0.0}]
    assert bench.served_max_diff(res, alone, None) == 2.0 ** -52
    # a sample: job k of the stream against the k-th job run alone
    assert bench.served_max_diff(res, alone[:2], [0, 1]) == 2.0 ** -52
    assert bench.served_max_diff(res[2:], alone[2:], None) is None  # failed jobs are not compared


def test_host_cpu_record():
    h = bench.host_cpu()
    assert h["nproc"] == os.cpu_count() and h["arch"]
    assert "model" not in h or isinstance(h["model"], str)
