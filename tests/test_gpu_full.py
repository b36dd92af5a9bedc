"""Full-size workloads against the oracle.

Two launch configurations:
* the one the benchmark times: ONE dim3_join_project call into caller-sized
  buffers on a fresh context (no counting call before it, so on the two-table
  workload the single emitting pass with look-back offsets runs);
* the plan path (dim3_partition, dim3_plan_row_counts, then
  dim3_plan_join_project / dim3_plan_join_count), which runs a counting pass
  and an emitting pass.

The oracle cannot produce 10^9+ pairs in seconds, so it recomputes sampled
rows one by one (its x filter): random rows, the first and last x, and the
rows that hold output positions 2^31 - 1, 2^31, 2^32 - 1 and 2^32 (where
32-bit offsets would wrap). Size and order are checked over the whole output.
"""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import check_sorted_distinct, dev, host, inst_dev, rows_of

pytestmark = pytest.mark.gpu


def closed_form_out_j(inst):
    """|OUT_J| = sum over y of deg_R(y) * deg_S(y) over distinct tuples."""
    ru = np.unique((inst.r_val.astype(np.int64) << 32) | (inst.r_key.astype(np.int64) & 0xFFFFFFFF))
    su = np.unique((inst.s_val.astype(np.int64) << 32) | (inst.s_key.astype(np.int64) & 0xFFFFFFFF))
    yr, cr = np.unique((ru & 0xFFFFFFFF).astype(np.uint32), return_counts=True)
    ys, cs = np.unique((su & 0xFFFFFFFF).astype(np.uint32), return_counts=True)
    _, ir, is_ = np.intersect1d(yr, ys, return_indices=True)
    return int((cr[ir].astype(np.int64) * cs[is_]).sum())


def sample_x(inst, k, seed):
    xs = np.unique(inst.r_val)
    rng = np.random.default_rng(seed)
    return np.concatenate([xs[:2], xs[-2:], rng.choice(xs, size=min(k, xs.size), replace=False)])


def boundary_x(out_x: torch.Tensor, total: int) -> np.ndarray:
    """x values of the rows holding output positions 0, total - 1 and the
    positions next to 2^31 and 2^32 that exist."""
    pos = [0, total - 1] + [p for b in (1 << 31, 1 << 32) for p in (b - 1, b) if p < total]
    idx = torch.tensor(sorted(set(p for p in pos if p >= 0)), dtype=torch.int64, device=out_x.device)
    return np.unique(host(out_x[idx]))


def run_one_call(inst, k_rows, single_pass: bool):
    """The benchmarked call: sizes from a separate plan on another context,
    then ONE dim3_join_project on a fresh context into buffers of exactly
    that size. Checks the count, order and distinctness on the device, and
    the sampled rows (random, first, last, around 2^31 and 2^32) against the
    oracle element by element."""
    cols = inst_dev(inst)
    sizing = dim3.Context(0)
    try:
        plan = sizing.partition(*cols)
        rc = host(plan.row_counts())
        dict_x = host(plan.export("dict_x"))
        plan.close()
    finally:
        sizing.close()
    total = int(rc.sum())
    ctx = dim3.Context(0)
    try:
        ctx.set_option(dim3.OPT_TIMING, 1)
        out_x = torch.empty(total, dtype=torch.int32, device="cuda")
        out_z = torch.empty(total, dtype=torch.int32, device="cuda")
        x, z = ctx.join_project(*cols, out_x=out_x, out_z=out_z)
        torch.cuda.synchronize()
        tm = ctx.timing()
        assert x.numel() == total
        if single_pass:
            assert ctx.last_path() == dim3.PATH_HYBRID
            assert tm["sparse_count"][1] == 0 and tm["sparse_emit"][1] >= 1, f"not one emitting pass: {tm}"
        check_sorted_distinct(x, z)
        xs = np.unique(np.concatenate([sample_x(inst, k_rows, 13), boundary_x(x, total)]))
        gx, gz, _ = rows_of(x, z, xs)
        ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val, x_filter=xs)
        assert gx.size == ox.size, f"{gx.size} sampled pairs vs oracle {ox.size}"
        assert np.array_equal(gx, ox) and np.array_equal(gz, oz)
        # every sampled row's size equals the separate plan's row count
        pos = np.searchsorted(dict_x, xs)
        present = (pos < dict_x.size) & (dict_x[np.minimum(pos, dict_x.size - 1)] == xs)
        ux, cnt = np.unique(ox, return_counts=True)
        exp = dict(zip(ux.tolist(), cnt.tolist()))
        for v, p in zip(xs[present], pos[present]):
            assert rc[p] == exp.get(int(v), 0), f"row of x={v}"
        del x, z, out_x, out_z
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def run_full(inst, k_rows, counts=False):
    ctx = dim3.Context(0)
    try:
        plan = ctx.partition(*inst_dev(inst))
        info = plan.info
        rc = plan.row_counts()
        total = int(rc.sum().item())
        if counts:
            x, z, c = plan.join_count()
        else:
            x, z = plan.join_project()
            c = None
        plan.close()
        torch.cuda.synchronize()
        assert x.numel() == total
        assert info["out_j"] == closed_form_out_j(inst)
        assert total <= info["out_j"]
        check_sorted_distinct(x, z)
        xs = sample_x(inst, k_rows, 11)
        gx, gz, gc = rows_of(x, z, xs, c)
        if counts:
            ox, oz, oc, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val, x_filter=xs)
            assert np.array_equal(gc, oc.astype(np.int32))
        else:
            ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val, x_filter=xs)
        assert np.array_equal(gx, ox) and np.array_equal(gz, oz)
        # per-row sizes of the sampled rows agree with row_counts
        dx = host(plan_dict_x(ctx, inst))
        pos = np.searchsorted(dx, np.unique(xs))
        present = (pos < dx.size) & (dx[np.minimum(pos, dx.size - 1)] == np.unique(xs))
        got = host(rc)[pos[present]]
        exp = np.array([(ox == v).sum() for v in np.unique(xs)[present]])
        assert np.array_equal(got, exp)
        del x, z, c
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def plan_dict_x(ctx, inst):
    plan = ctx.partition(*inst_dev(inst))
    d = plan.export("dict_x")
    plan.close()
    return d


def test_config2_one_call_single_pass():
    """|R| = |S| = 10^6, Zipf(1.0) y, ~5.0e9 pairs (output offsets past 2^32):
    the benchmarked one-call path (single emitting pass, look-back offsets),
    200 random rows plus the boundary rows exact."""
    run_one_call(gen.config2_two_table(), 200, single_pass=True)


def test_config3_one_call():
    """Chung-Lu 10^6 vertices, 4 x 10^6 edges, ~3.0e9 pairs (past 2^31): the
    benchmarked one-call path, 200 random rows plus the boundary rows exact."""
    run_one_call(gen.config3_chung_lu(), 200, single_pass=False)


def test_config2_full_sampled():
    """|R| = |S| = 10^6, Zipf(1.0) y: ~5e9 pairs through the plan path
    (counting pass, then emitting pass); 64 sampled rows exact."""
    run_full(gen.config2_two_table(), 64)


def test_config3_chung_lu_full_sampled():
    """Chung-Lu 10^6 vertices, 4 x 10^6 edges through the plan path: 200
    sampled rows exact (including hubs and leaves)."""
    run_full(gen.config3_chung_lu(), 200)


def test_config2_count_sampled_quarter():
    """Join-Count on a quarter-size two-table workload, sampled rows exact."""
    run_full(gen.config2_two_table(scale=0.25), 64, counts=True)
