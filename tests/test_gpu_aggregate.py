"""Parity of Join-Aggregate (Section 4.1) with the oracle: every aggregate and
function, bags with duplicate rows, several z tiles and many x. Integer
results are int64 and bit-exact; AVG is the float64 quotient of the same
int64 SUM and COUNT on both sides, so it is bit-exact too."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu

AGGS = {"count": dim3.AGG_COUNT, "sum": dim3.AGG_SUM, "min": dim3.AGG_MIN, "max": dim3.AGG_MAX,
        "avg": dim3.AGG_AVG}
FNS = {"mul": dim3.FN_MUL, "add": dim3.FN_ADD, "left": dim3.FN_LEFT, "right": dim3.FN_RIGHT}


@pytest.fixture(scope="module")
def ctx():
    c = dim3.Context(0)
    yield c
    c.close()


def _bag(seed, nr, ns, nx, ny, nz, vr=1000, zipf=None):
    rng = np.random.default_rng(seed)
    inst = gen.small_two_table(seed, n_r=nr, n_s=ns, nx=nx, ny=ny, nz=nz, zipf=zipf)
    # bags: repeat some rows, attach values
    r_rep = rng.integers(1, 3, inst.r_key.size)
    s_rep = rng.integers(1, 3, inst.s_key.size)
    r_key, r_val = np.repeat(inst.r_key, r_rep), np.repeat(inst.r_val, r_rep)
    s_key, s_val = np.repeat(inst.s_key, s_rep), np.repeat(inst.s_val, s_rep)
    r_v = rng.integers(-vr, vr, r_key.size).astype(np.int32)
    s_u = rng.integers(-vr, vr, s_key.size).astype(np.int32)
    return r_key, r_val, r_v, s_key, s_val, s_u


CASES = [
    dict(seed=31, nr=400, ns=400, nx=40, ny=30, nz=50),
    dict(seed=32, nr=6000, ns=5000, nx=700, ny=200, nz=5000, zipf=1.1),  # three z tiles
    dict(seed=33, nr=3000, ns=3000, nx=300, ny=40, nz=9000, vr=2**31 - 1),  # extreme values, wrapping sums
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("agg", list(AGGS))
@pytest.mark.parametrize("fn", list(FNS))
def test_join_aggregate_parity(ctx, case, agg, fn):
    cols = _bag(**CASES[case])
    ox, oz, ov = oracle.join_aggregate(*cols, agg, fn)
    x, z, v = ctx.join_aggregate(*[dev(c) for c in cols], AGGS[agg], FNS[fn])
    torch.cuda.synchronize()
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
    hv = host(v)
    assert hv.dtype == ov.dtype and np.array_equal(hv, ov)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("agg", list(AGGS))
def test_groupby_aggregate_parity(ctx, case, agg):
    r_key, r_val, _, s_key, s_val, _ = _bag(**CASES[case])
    ox, ov = oracle.groupby_aggregate(r_key, r_val, s_key, s_val, agg)
    x, v = ctx.groupby_aggregate(dev(r_key), dev(r_val), dev(s_key), dev(s_val), AGGS[agg])
    torch.cuda.synchronize()
    assert np.array_equal(host(x), ox) and np.array_equal(host(v), ov)


def test_aggregate_bench_tables_scaled(ctx):
    """The 1M x 1M Zipf tables at 2 %, with values: SUM of products."""
    inst = gen.config2_two_table(scale=0.02)
    rng = np.random.default_rng(5)
    r_v = rng.integers(-100, 100, inst.r_key.size).astype(np.int32)
    s_u = rng.integers(-100, 100, inst.s_key.size).astype(np.int32)
    cols = (inst.r_key, inst.r_val, r_v, inst.s_key, inst.s_val, s_u)
    ox, oz, ov = oracle.join_aggregate(*cols, "sum", "mul")
    x, z, v = ctx.join_aggregate(*[dev(c) for c in cols], dim3.AGG_SUM, dim3.FN_MUL)
    torch.cuda.synchronize()
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz) and np.array_equal(host(v), ov)


def test_aggregate_empty_and_errors(ctx):
    e = dev(np.zeros(0, np.int32))
    x, z, v = ctx.join_aggregate(e, e, e, e, e, e, dim3.AGG_SUM, dim3.FN_MUL)
    assert x.numel() == 0
    cols = [dev(c) for c in _bag(**CASES[0])]
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.join_aggregate(*cols, 9, dim3.FN_MUL)
    assert ei.value.status == -1
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.join_aggregate(*cols, dim3.AGG_SUM, 7)
    assert ei.value.status == -1
