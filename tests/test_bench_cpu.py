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


def test_cpu_baseline_checks_sampled_rows():
    """The oracle leg compares its rows with the same rows of a result (here a
    host copy of the oracle's own full result in CPU tensors), and flags a
    result with one wrong z; boundary rows of a short result are its first
    and last x."""
    import gen
    import oracle

    inst = gen.small_two_table(3, n_r=3000, n_s=2500, nx=300, ny=80, nz=250, zipf=1.0)
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    tx, tz = torch.from_numpy(ox.copy()), torch.from_numpy(oz.copy())
    bx = bench.boundary_x(torch, tx, ox.size)
    assert set(bx.tolist()) == {int(ox[0]), int(ox[-1])}
    base, ver = bench.cpu_baseline(inst, 0.01, check=(bx, lambda xs: bench.rows_on_device(torch, tx, tz, xs)))
    assert ver["ok"] and ver["rows"] >= 2 and base["kind"] == "oracle" and base["cores"] == 1
    tz[ox.size // 2] += 1
    mid = int(ox[ox.size // 2])
    _, ver = bench.cpu_baseline(inst, 0.01, check=(np.array([mid], np.int32),
                                                    lambda xs: bench.rows_on_device(torch, tx, tz, xs)))
    assert not ver["ok"]


def test_partition_roofline_formula():
    info = {"n_r": 100, "n_s": 50, "n_x": 10, "n_y": 5, "n_z": 7, "n_r_kept": 90}
    r = bench.partition_roofline(info, {"partition": 0.002}, 1000.0)
    alg = 16 * 150 + 4 * 22 + 12 * 140 + 8 * 17
    assert r["alg_bytes"] == alg and abs(r["achieved_gbs"] - alg / 2e-6 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved_gbs"] / 1000.0) < 1e-12
    assert bench.partition_roofline(info, {}, 1000.0)["frac"] is None


def test_host_region_info_finds_the_mapping():
    import mmap

    m = mmap.mmap(-1, 8 << 20, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    a = np.frombuffer(m, dtype=np.int32)
    a[:] = 1
    info = bench.host_region_info(a.ctypes.data)
    assert info["anon_huge_bytes"] is not None and info["anon_huge_bytes"] >= 0
    assert info["numa_pages"] is None or sum(info["numa_pages"].values()) >= 1


def test_sparse_passes_roofline_sums_both_passes():
    """The SparseBMM roofline of a step counts the counting (or staging) pass
    and the emitting pass together, per step, against the HBM peak."""
    tm = {"sparse_count": (40.0, 4), "sparse_emit": (10.0, 4)}
    peaks = {"hbm": 5000.0}
    r = bench.sparse_passes_roofline(tm, 2, 1e9, peaks)
    assert r["ms"] == 25.0
    assert abs(r["achieved_gbs"] - 1e9 / 0.025 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved_gbs"] / 5000.0) < 1e-12
    assert bench.sparse_passes_roofline({"sparse_count": (0.0, 0), "sparse_emit": (0.0, 0)}, 1, 1e9, peaks) is None
