"""Parity of the Section 2.2 mapping variants with the CPU oracle: skipped
mapping (pre-mapped ids, ``dim3_partition_ids``), multi-attribute mapping
(``dim3_map_tuples``) and id translation (``dim3_gather_i32``). Integer work:
bit-exact."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import dev, host
from tests.test_oracle_mapping_pins import composite_bruteforce

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = dim3.Context(0)
    yield c
    c.close()


def _tuples_case(seed, n, k, lo, hi, mask):
    rng = np.random.default_rng(seed)
    return [rng.integers(lo, hi, n).astype(np.int32) for _ in range(k)], mask


@pytest.mark.parametrize("seed,n,k,lo,hi,mask", [
    (1, 0, 1, 0, 1, 0),
    (2, 1, 3, -5, 5, 0),
    (3, 1000, 1, -2**31, 2**31 - 1, 0),
    (4, 1000, 1, -2**31, 2**31 - 1, 1),
    (5, 300_001, 2, -40, 40, 0),
    (6, 300_001, 2, -2**31, 2**31 - 1, 0b10),
    (7, 200_003, 4, -3, 3, 0b0101),
    (8, 100_000, 8, 0, 2, 0xFF),
    (9, 250_000, 3, 0, 1, 0),  # one distinct tuple
])
def test_map_tuples_parity(ctx, seed, n, k, lo, hi, mask):
    cols, mask = _tuples_case(seed, n, k, lo, hi, mask)
    oids, ofirst, od = oracle.map_tuples(cols, mask)
    ids, first = ctx.map_tuples([dev(c) for c in cols], mask)
    torch.cuda.synchronize()
    assert first.numel() == od
    assert np.array_equal(host(ids), oids) and np.array_equal(host(first), ofirst)


def test_map_tuples_all_distinct(ctx):
    rng = np.random.default_rng(10)
    v = rng.permutation(500_000).astype(np.int32) - 250_000
    ids, first = ctx.map_tuples([dev(v)])
    torch.cuda.synchronize()
    oids, ofirst, _ = oracle.map_tuples([v])
    assert np.array_equal(host(ids), oids) and np.array_equal(host(first), ofirst)


def _ids_instance(seed, nr, ns, n_x, n_y, n_z, neg_frac=0.0, zipf=None):
    rng = np.random.default_rng(seed)

    def col(n, m):
        if zipf:
            v = np.minimum(rng.zipf(zipf, n) - 1, m - 1)
            v = rng.permutation(m)[v]
        else:
            v = rng.integers(0, m, n)
        if neg_frac:
            v = np.where(rng.random(n) < neg_frac, -1 - rng.integers(0, 3, n), v)
        return v.astype(np.int32)

    return col(nr, n_y), col(nr, n_x), col(ns, n_y), col(ns, n_z)


@pytest.mark.parametrize("case", [
    dict(seed=1, nr=0, ns=0, n_x=0, n_y=0, n_z=0),
    dict(seed=2, nr=50, ns=0, n_x=10, n_y=10, n_z=10),
    dict(seed=3, nr=20_000, ns=20_000, n_x=3000, n_y=500, n_z=2000),
    dict(seed=4, nr=60_000, ns=60_000, n_x=5000, n_y=3000, n_z=70_000, neg_frac=0.05),
    dict(seed=5, nr=80_000, ns=80_000, n_x=4000, n_y=2000, n_z=30_000, zipf=1.2),
    dict(seed=6, nr=30_000, ns=30_000, n_x=100_000, n_y=200_000, n_z=450_000),  # sparse id ranges, z tiled
])
@pytest.mark.parametrize("theta", [-1, 8])
def test_partition_ids_parity(ctx, case, theta):
    r_y, r_x, s_y, s_z = _ids_instance(**{k: v for k, v in case.items() if k not in ("n_x", "n_y", "n_z")},
                                       n_x=max(case["n_x"], 1), n_y=max(case["n_y"], 1), n_z=max(case["n_z"], 1))
    plan = ctx.partition_ids(dev(r_y), dev(r_x), dev(s_y), dev(s_z), case["n_x"], case["n_y"], case["n_z"],
                             theta_z=theta)
    try:
        assert plan.info["n_x"] == case["n_x"] and plan.info["n_z"] == case["n_z"]
        x, z = plan.join_project()
        torch.cuda.synchronize()
        ox, oz, _ = oracle.join_project_ids(r_y, r_x, s_y, s_z)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        cx, cz, cc = plan.join_count()
        torch.cuda.synchronize()
        kx, kz, kc, _ = oracle.join_count_ids(r_y, r_x, s_y, s_z)
        assert np.array_equal(host(cx), kx) and np.array_equal(host(cz), kz)
        assert np.array_equal(host(cc), kc.astype(np.int32))
    finally:
        plan.close()


def test_partition_ids_matches_value_join(ctx):
    """The bench workload's tables, mapped by the oracle's rank map, give
    through the id path the rank-mapped value result."""
    inst = gen.config2_two_table(scale=0.02)
    yv = np.unique(inst.s_key)
    xv, zv = np.unique(inst.r_val), np.unique(inst.s_val)
    r_y = np.searchsorted(yv, inst.r_key).astype(np.int32)
    r_y[(r_y >= yv.size) | (yv[np.minimum(r_y, yv.size - 1)] != inst.r_key)] = -1  # y not in S.y
    r_x = np.searchsorted(xv, inst.r_val).astype(np.int32)
    s_y = np.searchsorted(yv, inst.s_key).astype(np.int32)
    s_z = np.searchsorted(zv, inst.s_val).astype(np.int32)
    plan = ctx.partition_ids(dev(r_y), dev(r_x), dev(s_y), dev(s_z), xv.size, yv.size, zv.size)
    try:
        x, z = plan.join_project()
        torch.cuda.synchronize()
    finally:
        plan.close()
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert np.array_equal(xv[host(x)], ox) and np.array_equal(zv[host(z)], oz)


@pytest.mark.parametrize("which", ["r_x", "r_y", "s_y", "s_z"])
def test_partition_ids_out_of_range(ctx, which):
    r_y, r_x, s_y, s_z = _ids_instance(7, 1000, 1000, 100, 50, 80)
    cols = dict(r_y=r_y, r_x=r_x, s_y=s_y, s_z=s_z)
    lim = dict(r_x=100, r_y=50, s_y=50, s_z=80)[which]
    cols[which] = cols[which].copy()
    cols[which][517] = lim
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.partition_ids(dev(cols["r_y"]), dev(cols["r_x"]), dev(cols["s_y"]), dev(cols["s_z"]), 100, 50, 80)
    assert ei.value.status == -1


def _composite_gpu(ctx, R, S):
    R = np.asarray(R, np.int32).reshape(-1, 4)
    S = np.asarray(S, np.int32).reshape(-1, 4)
    nr = R.shape[0]
    Rd = [dev(np.ascontiguousarray(R[:, i])) for i in range(4)]
    Sd = [dev(np.ascontiguousarray(S[:, i])) for i in range(4)]
    xid, xfirst = ctx.map_tuples([Rd[0], Rd[1]])
    yid, _ = ctx.map_tuples([torch.cat([Rd[2], Sd[0]]), torch.cat([Rd[3], Sd[1]])])
    zid, zfirst = ctx.map_tuples([Sd[0], Sd[1], Sd[2]])
    plan = ctx.partition_ids(yid[:nr].contiguous(), xid, yid[nr:].contiguous(), zid, xfirst.numel(),
                             int(yid.max().item()) + 1 if yid.numel() else 0, zfirst.numel())
    try:
        x, z = plan.join_project()
    finally:
        plan.close()
    xr, zr = ctx.gather(xfirst, x), ctx.gather(zfirst, z)
    out = [ctx.gather(Rd[0], xr), ctx.gather(Rd[1], xr), ctx.gather(Sd[0], zr), ctx.gather(Sd[1], zr),
           ctx.gather(Sd[2], zr)]
    torch.cuda.synchronize()
    return np.stack([host(o) for o in out], axis=1) if x.numel() else np.zeros((0, 5), np.int32)


@pytest.mark.parametrize("seed", range(4))
def test_composite_example_gpu(ctx, seed):
    """Section 2.2's Pi_{a,b,c,d,e}(R(a,b,c,d) join_{c,d} S(c,d,e,f)) through
    map_tuples, partition_ids, the join and gather, against nested loops."""
    rng = np.random.default_rng(500 + seed)
    n = 60 if seed < 2 else 400
    R = [tuple(int(v) for v in rng.integers(-3, 4, 4)) for _ in range(n)]
    S = [tuple(int(v) for v in rng.integers(-3, 4, 4)) for _ in range(n)]
    got = [tuple(int(v) for v in row) for row in _composite_gpu(ctx, R, S)]
    assert got == composite_bruteforce(R, S)


def test_composite_larger_vs_oracle_flow(ctx):
    from tests.test_oracle_mapping_pins import composite_via_ids

    rng = np.random.default_rng(600)
    R = rng.integers(-20, 20, (30_000, 4)).astype(np.int32)
    S = rng.integers(-20, 20, (30_000, 4)).astype(np.int32)
    R[:, 2:] = rng.integers(0, 6, (30_000, 2))
    S[:, :2] = rng.integers(0, 6, (30_000, 2))
    got = [tuple(int(v) for v in row) for row in _composite_gpu(ctx, R, S)]
    assert got == composite_via_ids(R, S)


def test_gather_out_of_range(ctx):
    src = dev(np.arange(10, dtype=np.int32))
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.gather(src, dev(np.array([0, 3, 10], np.int32)))
    assert ei.value.status == -1
    out = ctx.gather(src, dev(np.array([9, 0, 4], np.int32)))
    torch.cuda.synchronize()
    assert host(out).tolist() == [9, 0, 4]
