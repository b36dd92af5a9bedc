"""Host-side pieces of bench.py that need no GPU: column placement for
self-joins, the stored traffic figure's bookkeeping, and argument defaults."""

import json
import os

import numpy as np
import torch

import bench


def test_device_columns_share_repeated_arrays():
    a = np.arange(10, dtype=np.int32)
    b = np.arange(10, 20, dtype=np.int32)
    cols = bench.device_columns(torch, [a, b, a, b], "cpu")
    assert cols[0] is cols[2] and cols[1] is cols[3]
    assert cols[0] is not cols[1]
    assert torch.equal(cols[0], torch.from_numpy(a)) and torch.equal(cols[1], torch.from_numpy(b))


def test_device_columns_copies_distinct_arrays():
    a = np.arange(5, dtype=np.int32)
    cols = bench.device_columns(torch, [a, a.copy(), a, a.copy()], "cpu")
    assert cols[0] is cols[2]
    assert cols[1] is not cols[3] and cols[0] is not cols[1]


def test_traffic_entry_bookkeeping():
    """Every stored traffic figure names an existing source file and scales
    consistently (DRAM bytes of the full launch = small capture x scale)."""
    p = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(p) as f:
        d = json.load(f)
    assert d, "no traffic entries"
    for wl, e in d.items():
        assert wl in bench.WORKLOADS
        src = os.path.join(bench.ROOT, "paper_2206_04995_gb300", "csrc", e["source"])
        assert os.path.exists(src)
        assert len(e["source_sha"]) == 16
        assert abs(e["dram_bytes_per_launch_small"] * e["scale"] - e["dram_bytes_per_launch_full"]) <= 1e-6 * \
            e["dram_bytes_per_launch_full"] + 1
        # algorithmic bytes are exact per workload (8 B per pair plus the R and S
        # columns, which do not scale with the pairs), so they agree only roughly
        assert abs(e["alg_bytes_per_launch_small"] * e["scale"] / e["alg_bytes_per_launch_full"] - 1) < 0.01
        # DRAM traffic of the emitting kernel cannot fall far below the bytes it must write
        assert 0.9 <= e["dram_bytes_per_launch_full"] / e["alg_bytes_per_launch_full"] <= 1.5


def test_traffic_for_unknown_workload():
    assert bench.traffic_for("no_such_workload") == (None, None)


def test_default_arguments(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py"])
    args = bench.parse_args()
    assert args.gpus == 1 and args.warmup >= 3 and args.steps >= 1
    assert args.workload == "two_table_1m_zipf1" and args.impl == "ours"
    assert not args.f1_sweep and not args.no_e2e
