"""Join-Count (COUNT per (x, z) pair) of single instances against the oracle,
exactly: every counter width the library picks from the largest |R[x]| (8
bits up to 255 R entries, 16 up to 65,535, else 32), one and several z
tiles, DenseEC counts added in, x ranges of a plan and unaligned output
buffers."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import host, inst_dev

pytestmark = pytest.mark.gpu


def _wide_hub(seed, n_hub_y):
    """One x joined with n_hub_y distinct y (|R[x]| above 65,535 when
    n_hub_y is), plus small random rows; S over a few thousand z."""
    rng = np.random.default_rng(seed)
    ys = np.arange(n_hub_y, dtype=np.int64) * 7 - 10**6
    r_key = np.concatenate([ys, rng.choice(ys, 20_000)]).astype(np.int32)
    r_val = np.concatenate([np.full(n_hub_y, -5, np.int64), rng.integers(-10**6, 10**6, 20_000)]).astype(np.int32)
    s_key = rng.choice(ys, 150_000).astype(np.int32)
    s_val = rng.integers(0, 3000, 150_000).astype(np.int32)
    return gen.Instance("hub", r_key, r_val, s_key, s_val)


CASES = {
    "cb8_multi_tile": lambda: gen.small_two_table(31, n_r=60_000, n_s=60_000, nx=6000, ny=2000, nz=200_000),
    # 28,000 z: one tile of ~7,000 counter words, the largest shared-memory footprint
    "cb8_largest_tile": lambda: gen.small_two_table(37, n_r=3000, n_s=200_000, nx=500, ny=2000, nz=28_000),
    "cb8_one_tile": lambda: gen.small_two_table(32, n_r=40_000, n_s=40_000, nx=4000, ny=1000, nz=3000, zipf=0.8),
    "cb16_multi_tile": lambda: gen.small_two_table(33, n_r=40_000, n_s=40_000, nx=50, ny=5000, nz=60_000, zipf=1.0),
    "cb16_power_law": lambda: gen.chung_lu_self(np.random.default_rng(34), 60_000, 80_000, 2.1),
    "cb32_hub": lambda: _wide_hub(35, 70_000),
    "duplicates": lambda: gen.small_two_table(36, n_r=5000, n_s=5000, nx=300, ny=100, nz=400, dup_frac=0.3),
}


@pytest.fixture(scope="module")
def cases():
    out = {}
    for name, make in CASES.items():
        inst = make()
        out[name] = (inst, *oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[:3])
    return out


def ctx_with(opts):
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, dim3.PATH_HYBRID)
    for k, v in opts.items():
        c.set_option(k, v)
    return c


@pytest.mark.parametrize("name", list(CASES))
def test_count_vs_oracle(name, cases):
    inst, ox, oz, oc = cases[name]
    c = ctx_with({})
    try:
        cols = inst_dev(inst)
        bx = torch.empty(ox.size + 7, dtype=torch.int32, device="cuda")
        bz = torch.empty(ox.size + 7, dtype=torch.int32, device="cuda")
        bc = torch.empty(ox.size + 7, dtype=torch.int32, device="cuda")
        x, z, cnt = c.join_count(*cols, out_x=bx[1:], out_z=bz[2:], out_c=bc[3:])
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), name
        assert np.array_equal(host(cnt), oc.astype(np.int32)), name
        plan = c.partition(*cols)
        n_x = plan.info["n_x"]
        parts = [plan.join_count(a, b) for a, b in ((0, n_x // 3), (n_x // 3, n_x // 3), (n_x // 3, n_x))]
        plan.close()
        for i, o in ((0, ox), (1, oz), (2, oc.astype(np.int32))):
            assert np.array_equal(np.concatenate([host(p[i]) for p in parts]), o), name
    finally:
        c.close()


@pytest.mark.parametrize("variant", [dim3.DENSE_TC, dim3.DENSE_POPC, dim3.DENSE_PROBE])
def test_count_with_dense_part(variant, cases):
    """DenseEC's per-pair counts added into the packed counters."""
    c = ctx_with({dim3.OPT_THETA_Z: 8, dim3.OPT_DENSE_VARIANT: variant})
    try:
        for name in ("cb8_multi_tile", "cb16_multi_tile", "cb16_power_law"):
            inst, ox, oz, oc = cases[name]
            x, z, cnt = c.join_count(*inst_dev(inst))
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), name
            assert np.array_equal(host(cnt), oc.astype(np.int32)), name
    finally:
        c.close()
