"""Parity of partial result caching (Section 3) with the oracle: the cache's
entries (selection by CacheScore under a budget, lists and complements) and
the results of plans built with a cache (which must equal the full result).
Integer work and float64 scores computed the same way on both sides:
bit-exact."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import dev, host, inst_dev

pytestmark = pytest.mark.gpu

BIG = 2**31 - 1


@pytest.fixture(scope="module")
def ctx():
    c = dim3.Context(0)
    yield c
    c.close()


def _instances():
    return [
        gen.small_two_table(21, n_r=3000, n_s=3000, nx=200, ny=80, nz=150, zipf=1.1),
        gen.small_two_table(22, n_r=8000, n_s=6000, nx=1000, ny=300, nz=2000, zipf=1.3),
        gen.chung_lu_self(np.random.default_rng(23), 5000, 20_000, 2.1),
    ]


def _check_cache(ctx, inst, theta, budget, ts, td):
    oc = oracle.cache_build(inst.r_key, inst.r_val, inst.s_key, inst.s_val, theta, budget, ts, td)
    c = ctx.cache_build(*inst_dev(inst), budget, theta_z=theta, t_sparse=ts, t_dense=td)
    try:
        e = c.export()
        torch.cuda.synchronize()
        info = c.info
        assert info["n_x"] == oc.n_x and info["n_entries"] == oc.z.size and info["n_list"] == oc.xs.size
        ks = [int(sz) + oc.n_x if cp else int(sz) for sz, cp in zip(oc.size, oc.complement)]
        space = sum(2 + min(k, oc.n_x - k) for k in ks)
        assert info["space"] == space <= budget
        assert np.array_equal(host(e["z"]), oc.z)
        assert np.array_equal(host(e["size"]), oc.size)
        assert np.array_equal(host(e["complement"]).astype(bool), oc.complement)
        assert np.array_equal(host(e["offsets"]), oc.offsets)
        assert np.array_equal(host(e["xs"]), oc.xs)
    except BaseException:
        c.close()
        raise
    return c, oc


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("theta,budget,ts,td", [
    (BIG, 0, 1.0, 1.0),
    (BIG, 50, 1.0, 1.0),
    (BIG, 5000, 1.2e-12, 1.1e-11),
    (8, 5000, 1.0, 0.5),
    (8, 10**12, 1.0, 0.01),
])
def test_cache_entries_parity(ctx, which, theta, budget, ts, td):
    inst = _instances()[which]
    c, _ = _check_cache(ctx, inst, theta, budget, ts, td)
    c.close()


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("theta,variant", [(BIG, 0), (8, dim3.DENSE_TC), (8, dim3.DENSE_POPC), (8, dim3.DENSE_PROBE)])
@pytest.mark.parametrize("budget", [0, 3000, 10**12])
def test_cached_plan_gives_full_result(ctx, which, theta, variant, budget):
    inst = _instances()[which]
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    c = ctx.cache_build(*inst_dev(inst), budget, theta_z=theta, t_sparse=1.0, t_dense=0.3)
    ctx.set_option(dim3.OPT_DENSE_VARIANT, variant)
    try:
        plan = ctx.partition_cached(*inst_dev(inst), c, theta_z=theta)
        try:
            assert plan.info["n_z_cached"] == c.info["n_entries"]
            x, z = plan.join_project()
            torch.cuda.synchronize()
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
            # x-range chunks concatenate into the same result
            n_x = plan.info["n_x"]
            cuts = [0, n_x // 3, n_x // 3 + 1, n_x]
            xs, zs = [], []
            for a, b in zip(cuts, cuts[1:]):
                cx, cz = plan.join_project(a, b)
                xs.append(host(cx))
                zs.append(host(cz))
            assert np.array_equal(np.concatenate(xs), ox) and np.array_equal(np.concatenate(zs), oz)
        finally:
            plan.close()
    finally:
        ctx.set_option(dim3.OPT_DENSE_VARIANT, 0)
        c.close()


@pytest.mark.parametrize("two_pass", [0, 1])
def test_cached_one_call_buffers(ctx, two_pass):
    """Caller-sized buffers (single-pass emission where it applies)."""
    inst = _instances()[1]
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    c = ctx.cache_build(*inst_dev(inst), 20_000, t_sparse=1.0, t_dense=1.0)
    ctx.set_option(dim3.OPT_TWO_PASS, two_pass)
    try:
        plan = ctx.partition_cached(*inst_dev(inst), c)
        bx = torch.empty(ox.size + 3, dtype=torch.int32, device="cuda")
        bz = torch.empty(ox.size + 3, dtype=torch.int32, device="cuda")
        x, z = plan.join_project(out_x=bx, out_z=bz)
        torch.cuda.synchronize()
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        plan.close()
    finally:
        ctx.set_option(dim3.OPT_TWO_PASS, 0)
        c.close()


def test_cached_plan_rejects_count(ctx):
    inst = _instances()[0]
    c = ctx.cache_build(*inst_dev(inst), 1000, t_sparse=1.0, t_dense=1.0)
    plan = ctx.partition_cached(*inst_dev(inst), c)
    try:
        with pytest.raises(dim3.Dim3Error) as ei:
            plan.join_count()
        assert ei.value.status == -7
    finally:
        plan.close()
        c.close()


def test_cache_on_other_tables_rejected(ctx):
    a, b = _instances()[0], _instances()[1]
    c = ctx.cache_build(*inst_dev(a), 10**9, t_sparse=1.0, t_dense=1.0)
    try:
        with pytest.raises(dim3.Dim3Error) as ei:
            ctx.partition_cached(*inst_dev(b), c)
        assert ei.value.status == -1
    finally:
        c.close()


def test_cache_bad_arguments(ctx):
    inst = _instances()[0]
    for kw in (dict(budget=-1), dict(budget=10, t_sparse=-1.0), dict(budget=10, t_dense=float("nan"))):
        budget = kw.pop("budget")
        with pytest.raises(dim3.Dim3Error) as ei:
            ctx.cache_build(*inst_dev(inst), budget, **kw)
        assert ei.value.status == -1


def test_cache_bench_workload_scaled(ctx):
    """The 1M x 1M Zipf tables at 2 %: entries and the cached result."""
    inst = gen.config2_two_table(scale=0.02)
    c, oc = _check_cache(ctx, inst, BIG, inst.nr + inst.ns, dim3.Context.T_SPARSE, dim3.Context.T_DENSE)
    try:
        plan = ctx.partition_cached(*inst_dev(inst), c)
        x, z = plan.join_project()
        torch.cuda.synchronize()
        plan.close()
        ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        assert oc.z.size > 0
    finally:
        c.close()
