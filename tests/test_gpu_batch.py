"""Batched execution: every instance of a batch gets exactly its own result
(oracle per instance, and the single-instance CUDA path), whatever the other
instances hold -- including the same values, which must not join across
instances."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import dev, host, inst_dev, rows_of

pytestmark = pytest.mark.gpu


def ctx_with(opts=None):
    c = dim3.Context(0)
    for k, v in (opts or {}).items():
        c.set_option(k, v)
    return c


def split(arr, counts):
    out, a = [], 0
    for c in counts:
        out.append(arr[a:a + c])
        a += c
    return out


def check_batch(c, insts, counts_mode=False):
    cols = [inst_dev(i) for i in insts]
    if counts_mode:
        x, z, cnt, per = c.batch_join_count(cols)
        xs, zs, cs = split(host(x), per), split(host(z), per), split(host(cnt), per)
    else:
        x, z, per = c.batch_join_project(cols)
        xs, zs = split(host(x), per), split(host(z), per)
    assert sum(per) == x.numel()
    for t, inst in enumerate(insts):
        if counts_mode:
            ox, oz, oc, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
            assert np.array_equal(cs[t], oc.astype(np.int32)), f"instance {t} counts"
        else:
            ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
        assert per[t] == ox.size, f"instance {t}: {per[t]} vs {ox.size}"
        assert np.array_equal(xs[t], ox) and np.array_equal(zs[t], oz), f"instance {t}"


def mixed_batch(seed, k=12):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        nx, ny, nz = (int(v) for v in rng.integers(1, 200, size=3))
        out.append(gen.small_two_table(seed * 100 + i, n_r=int(rng.integers(0, 3000)), n_s=int(rng.integers(0, 3000)),
                                       nx=nx, ny=ny, nz=nz, zipf=[None, 1.0][i % 2], dup_frac=0.1 * (i % 3 == 0),
                                       self_join=(i % 4 == 3)))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_batch_mixed(seed):
    c = ctx_with()
    insts = mixed_batch(seed)
    check_batch(c, insts)
    check_batch(c, insts, counts_mode=True)
    c.close()


def test_batch_same_values_do_not_join_across_instances():
    base = gen.small_two_table(5, n_r=2000, n_s=1800, nx=100, ny=60, nz=90, zipf=1.0)
    other = gen.small_two_table(6, n_r=1500, n_s=1500, nx=80, ny=50, nz=70, zipf=1.0)
    # instance 2 uses base's y values with other x/z: joins with base's S must not appear
    mixed = gen.Instance("mix", r_key=base.r_key[:900], r_val=other.r_val[:900], s_key=other.s_key, s_val=other.s_val)
    insts = [base, base, mixed, other, base]
    c = ctx_with()
    check_batch(c, insts)
    check_batch(c, insts, counts_mode=True)
    c.close()


def test_batch_with_empty_instances():
    e = np.zeros(0, np.int32)
    insts = [gen.Instance("e", e, e, e, e), gen.small_two_table(1, n_r=500, n_s=500, nx=40, ny=30, nz=35),
             gen.Instance("no_s", np.array([1], np.int32), np.array([2], np.int32), e, e),
             gen.small_two_table(2, n_r=700, n_s=600, nx=50, ny=20, nz=45, zipf=1.1),
             gen.Instance("e2", e, e, e, e)]
    c = ctx_with()
    check_batch(c, insts)
    c.close()


@pytest.mark.parametrize("variant", [dim3.DENSE_TC, dim3.DENSE_POPC, dim3.DENSE_PROBE])
@pytest.mark.parametrize("theta", [0, 6])
def test_batch_dense_variants(variant, theta):
    """Block-diagonal DenseEC: tiles that straddle instances stay correct."""
    c = ctx_with({dim3.OPT_THETA_Z: theta, dim3.OPT_DENSE_VARIANT: variant})
    insts = mixed_batch(10 + variant, k=9) + [gen.small_two_table(77, n_r=20_000, n_s=16_000, nx=700, ny=300,
                                                                   nz=500, zipf=0.9)]
    check_batch(c, insts)
    check_batch(c, insts, counts_mode=True)
    c.close()


def test_batch_wide_rows_windowed():
    """Wide S_sparse rows (bitmaps over each instance's own z window)."""
    c = ctx_with({dim3.OPT_BITMAP_ROW_MIN: 1})
    check_batch(c, mixed_batch(21, k=10))
    c.close()


def test_batch_config4_scaled_vs_oracle():
    insts = gen.config4_batch(n_inst=24, lo=1000, hi=20_000)
    c = ctx_with()
    check_batch(c, insts)
    c.close()


def test_batch_config4_full_vs_single_path():
    """The 256-instance workload: every instance equals the one-at-a-time path;
    the 6 smallest instances are checked against the oracle whole, and the 8
    largest (up to ~3e8 pairs each) on 48 sampled x rows each (the first, the
    last and random ones) through the oracle's x filter."""
    insts = gen.config4_batch()
    c = ctx_with()
    cols = [inst_dev(i) for i in insts]
    x, z, per = c.batch_join_project(cols)
    off = np.concatenate([[0], np.cumsum(per)])
    order = sorted(range(len(insts)), key=lambda t: insts[t].nr)
    small, large = order[:6], order[-8:]
    rng = np.random.default_rng(41)
    for t, col in enumerate(cols):
        sx, sz = c.join_project(*col)
        assert per[t] == sx.numel()
        bx, bz = x[off[t]:off[t + 1]], z[off[t]:off[t + 1]]
        assert torch.equal(bx, sx) and torch.equal(bz, sz), f"instance {t}"
        i = insts[t]
        if t in small:
            ox, oz, _ = oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)
            assert np.array_equal(host(sx), ox) and np.array_equal(host(sz), oz)
        if t in large:
            xs = np.unique(i.r_val)
            pick = np.unique(np.concatenate([xs[:1], xs[-1:], rng.choice(xs, size=46, replace=False)]))
            gx, gz, _ = rows_of(bx, bz, pick)
            ox, oz, _ = oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val, x_filter=pick)
            assert gx.size == ox.size, f"instance {t}: sampled rows {gx.size} vs oracle {ox.size}"
            assert np.array_equal(gx, ox) and np.array_equal(gz, oz), f"instance {t} sampled rows"
    c.close()


def test_batch_plan_ranges_and_preallocated_call():
    insts = mixed_batch(3, k=7)
    c = ctx_with()
    cols = [inst_dev(i) for i in insts]
    plan = c.batch_partition(cols)
    lo = plan.instance_ranges()
    assert lo[0] == 0 and lo[-1] == plan.info["n_x"] and all(a <= b for a, b in zip(lo, lo[1:]))
    parts = [plan.join_project(lo[t], lo[t + 1]) for t in range(len(insts))]
    plan.close()
    n = sum(p[0].numel() for p in parts)
    bx = torch.empty(n + 5, dtype=torch.int32, device="cuda")
    bz = torch.empty(n + 5, dtype=torch.int32, device="cuda")
    x, z, per = c.batch_join_project(cols, out_x=bx[1:], out_z=bz[3:])
    assert per == [p[0].numel() for p in parts]
    assert torch.equal(x, torch.cat([p[0] for p in parts])) and torch.equal(z, torch.cat([p[1] for p in parts]))
    with pytest.raises(dim3.Dim3Error):
        c.batch_join_project(cols, out_x=bx[: n - 1], out_z=bz[: n - 1])
    c.close()


@pytest.mark.parametrize("rows", [1, 2, 4])
@pytest.mark.parametrize("two_pass", [0, 1])
def test_batch_rows_per_cta(rows, two_pass):
    """Batches emitted with 1, 2 or 4 x rows per CTA (groups that never cross
    an instance, ragged at every instance end), one pass and two, with wide
    S rows held as bitmaps over each instance's window and DenseEC results
    over each instance's dense index."""
    for opts in ({}, {dim3.OPT_BITMAP_ROW_MIN: 1}, {dim3.OPT_THETA_Z: 6, dim3.OPT_DENSE_VARIANT: dim3.DENSE_POPC}):
        c = ctx_with({dim3.OPT_EMIT_ROWS: rows, dim3.OPT_TWO_PASS: two_pass, **opts})
        insts = mixed_batch(31 + rows, k=11) + gen.config4_batch(n_inst=5, lo=1000, hi=15_000)
        cols = [inst_dev(i) for i in insts]
        n = sum(oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)[0].size for i in insts)
        bx = torch.empty(n + 3, dtype=torch.int32, device="cuda")
        bz = torch.empty(n + 3, dtype=torch.int32, device="cuda")
        x, z, per = c.batch_join_project(cols, out_x=bx[1:], out_z=bz[2:])
        off = np.concatenate([[0], np.cumsum(per)])
        for t, i in enumerate(insts):
            ox, oz, _ = oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)
            assert np.array_equal(host(x[off[t]:off[t + 1]]), ox), (rows, two_pass, opts, t)
            assert np.array_equal(host(z[off[t]:off[t + 1]]), oz), (rows, two_pass, opts, t)
        c.close()
