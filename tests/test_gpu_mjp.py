"""Multi-way joins with projection (Section 4.2) on the GPU against the
oracle: exact chain sizes, every deduplication placement of short chains, and
the DP's placement on a power-law graph. Integer work: bit-exact."""

import itertools

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = dim3.Context(0)
    yield c
    c.close()


def rand_tables(seed, k, n, span):
    rng = np.random.default_rng(seed)
    return [(rng.integers(-span, span, n).astype(np.int32), rng.integers(-span, span, n).astype(np.int32))
            for _ in range(k)]


def on_dev(tables):
    return [(dev(a), dev(b)) for a, b in tables]


@pytest.mark.parametrize("seed,k,n,span", [(1, 1, 50, 5), (2, 2, 500, 30), (3, 3, 2000, 200), (4, 4, 3000, 400)])
def test_sizes_parity(ctx, seed, k, n, span):
    tables = rand_tables(seed, k, n, span)
    oj, op = oracle.chain_sizes(tables)
    gj, gp = ctx.mjp_sizes(on_dev(tables))
    assert gj == oj and gp == op


@pytest.mark.parametrize("seed,k,n,span", [(5, 2, 800, 40), (6, 3, 2000, 150), (7, 4, 3000, 300)])
def test_every_placement(ctx, seed, k, n, span):
    tables = rand_tables(seed, k, n, span)
    ox, oz = oracle.line_join_project(tables)
    dt = on_dev(tables)
    for middle in itertools.product([0, 1], repeat=k - 2):
        x, z = ctx.mjp_execute(dt, [0, *middle, 1])
        torch.cuda.synchronize()
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), middle


def test_three_hop_power_law(ctx):
    """Pi_{x_1, x_4}(E join E join E) on a capped Chung-Lu graph: sizes, the
    DP's placement, and the result against the oracle."""
    g = gen.chung_lu_self(np.random.default_rng(8), 8000, 16_000, 2.1)
    edges = (g.r_val, g.r_key)  # R(x, y): the edge x -> y
    tables = [edges] * 3
    oj, op = oracle.chain_sizes(tables)
    dt = on_dev(tables)
    gj, gp = ctx.mjp_sizes(dt)
    assert gj == oj and gp == op
    r_size = [float(np.unique(np.stack(edges, 1), axis=0).shape[0])] * 3
    dedup, cost = dim3.Context.mjp_plan(r_size, gj, gp)
    ocost, odedup = oracle.mjp_dp(r_size, oj, op, list(dim3.Context.MJP_COSTS))
    assert dedup == odedup and cost == pytest.approx(ocost, rel=1e-12)
    ox, oz = oracle.line_join_project(tables)
    x, z = ctx.mjp_execute(dt, dedup)
    torch.cuda.synchronize()
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)


def test_mjp_errors(ctx):
    dt = on_dev(rand_tables(9, 3, 100, 10))
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.mjp_execute(dt, [0, 1, 0])
    assert ei.value.status == -1
    ox, _ = oracle.line_join_project(rand_tables(9, 3, 100, 10))
    bx = torch.empty(max(ox.size - 1, 0), dtype=torch.int32, device="cuda")
    bz = torch.empty(max(ox.size - 1, 0), dtype=torch.int32, device="cuda")
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.mjp_execute(dt, [0, 0, 1], out=(bx, bz))
    assert ei.value.status == -4
