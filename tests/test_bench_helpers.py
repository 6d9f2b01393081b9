"""Host-side helpers of bench.py: the kernel named for each route of a plan
description, the chain labels of the JSON line, and the DRAM-traffic
records, which are used only while every source file they were taken from
is unchanged (one file or several, hashed in order)."""
import hashlib
import json
import os

import numpy as np

import bench


def test_kernel_name_per_route():
    assert bench.kernel_name({"kind": "chain_fft", "M": 16384}) == "k_fir_fft"
    assert bench.kernel_name({"kind": "fir_fft", "P": 0}) == "k_fir_fft"
    assert bench.kernel_name({"kind": "fir_fft", "P": 2}) == "k_fir_fft_spec+k_fir_fft_conv"
    assert bench.kernel_name({"kind": "fir_tc", "kernel": "k_fir_tc_ws"}) == "k_fir_tc_ws"
    assert bench.kernel_name({"kind": "cascade", "scan": "tc"}) == "k_sos_tc"
    assert bench.kernel_name({"kind": "cascade", "scan": "warp"}) == "k_sos_warp"
    assert bench.kernel_name({"kind": "cascade", "scan": "block"}) == "k_unit"
    assert bench.kernel_name({"kind": "fused", "S": 2, "L": 31}) == "k_unit"


def test_chain_label():
    st = [("sos", np.zeros((2, 6))), ("fir", np.zeros(101)), ("sos", np.zeros((1, 6)))]
    assert bench.chain_label(st) == "2 SOS + FIR 101 + 1 SOS"
    assert bench.chain_label([]) == ""


def test_traffic_records_follow_their_sources(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "src").mkdir()
    a, b = root / "src" / "a.cu", root / "src" / "b.cuh"
    a.write_text("kernel a\n")
    b.write_text("header b\n")

    def h(*paths):
        d = hashlib.sha256()
        for p in paths:
            d.update(p.read_bytes())
        return d.hexdigest()[:16]

    rec = {"k_one": {"w": {"source": "src/a.cu", "source_sha256_16": h(a), "dram_bytes_per_launch": 100.0}},
           "k_two": {"w": {"source": ["src/a.cu", "src/b.cuh"], "source_sha256_16": h(a, b),
                           "dram_bytes_per_launch": 200.0}},
           "k_order": {"w": {"source": ["src/b.cuh", "src/a.cu"], "source_sha256_16": h(a, b),
                             "dram_bytes_per_launch": 300.0}}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_for("k_one", "w") == 100.0
    assert bench.traffic_for("k_two", "w") == 200.0
    assert bench.traffic_for("k_order", "w") is None  # hashed in the listed order
    assert bench.traffic_for("k_one", "other") is None
    assert bench.traffic_for("k_none", "w") is None
    b.write_text("header b, changed\n")  # a shared header changed: the two-file record is stale
    assert bench.traffic_for("k_one", "w") == 100.0
    assert bench.traffic_for("k_two", "w") is None
    os.remove(a)
    assert bench.traffic_for("k_one", "w") is None
