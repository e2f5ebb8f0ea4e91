"""Host-side measurement logic of bench.py, on the CPU: the algorithmic
bytes of the roofline (each root's DAG row and its candidates' rows, for the
roots that can hold a k-clique), plan parsing, the reading of nvidia-smi
clock samples (a throttle reason is reported, a missing sample is not
invented), whole-job throughput of replicas, and the guard that drops ncu
counters taken on other kernel sources."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2104_13209_gb300 import synth  # noqa: E402


def _bytes_by_loop(drp, dci, k):
    total = 0
    for v in range(len(drp) - 1):
        row = dci[drp[v]:drp[v + 1]]
        if len(row) < k - 1:
            continue
        total += 4 * len(row)
        for u in row:
            total += 4 * int(drp[u + 1] - drp[u])
    return total


def test_algorithmic_bytes_match_the_definition():
    g = synth.rmat(10, 8, seed=5)
    drp, dci, _, _ = O.dag_for(g.row_ptr, g.col_idx, "degeneracy")
    for k in (3, 4, 6):
        assert bench.algorithmic_bytes(drp, dci, k) == _bytes_by_loop(drp, dci, k)
    # a star oriented away from its centre: one root with every leaf as a
    # candidate, and no leaf row
    rp = np.array([0, 4, 4, 4, 4, 4], dtype=np.uint32)
    ci = np.array([1, 2, 3, 4], dtype=np.uint32)
    assert bench.algorithmic_bytes(rp, ci, 4) == 16
    assert bench.algorithmic_bytes(rp, ci, 6) == 0


def test_parse_plan():
    assert bench.parse_plan("4vc,4ec") == [(4, "vc"), (4, "ec")]
    assert bench.parse_plan(" 7 ") == [(7, "vc")]


def test_clock_summary_reports_reasons_and_medians():
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbled",
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_replica_throughput_and_single_rank_max():
    assert bench.replica_throughput(10.0, 2.0, 4) == 20.0
    assert bench.max_over_ranks(3.5) == 3.5


def test_counters_of_other_sources_are_dropped(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.traffic_record() == {}
    rec = {"kernel_source_sha256_16": "0" * 16, "dram_bytes_per_launch": 1}
    (tmp_path / "traffic.json").write_text(json.dumps(rec))
    assert bench.traffic_record() == {}
    rec["kernel_source_sha256_16"] = bench.kernel_source_hash()
    (tmp_path / "traffic.json").write_text(json.dumps(rec))
    assert bench.traffic_record()["dram_bytes_per_launch"] == 1
