"""Tensor-core DenseEC (Algorithm 3 as a 0/1 product) at both tile widths the
tuner chooses between (128 x 256 and 128 x 128 tiles of C), against the
oracle exactly: several raster groups of row tiles (more than 16 row tiles,
a ragged last group), ragged column tiles, counts (Join-Count) as well as
pairs, and a batch's block-diagonal tile list."""

import numpy as np
import pytest

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import host, inst_dev

pytestmark = pytest.mark.gpu


def ctx_with(opts):
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, dim3.PATH_HYBRID)
    for k, v in opts.items():
        c.set_option(k, v)
    return c


@pytest.fixture(scope="module")
def wide():
    # 3,000 x rows: 24 row tiles of 128 (a full raster group of 16 and a
    # ragged one of 8); 700 dense z: 3 or 6 column tiles with a ragged edge
    inst = gen.small_two_table(51, n_r=90_000, n_s=60_000, nx=3000, ny=900, nz=700, zipf=0.9)
    return inst, *oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[:3]


@pytest.mark.parametrize("tile_n", [128, 256])
def test_tc_tile_widths(tile_n, wide):
    inst, ox, oz, oc = wide
    c = ctx_with({dim3.OPT_THETA_Z: 0, dim3.OPT_DENSE_VARIANT: dim3.DENSE_TC, dim3.OPT_DENSE_TILE_N: tile_n})
    try:
        cols = inst_dev(inst)
        x, z = c.join_project(*cols)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        x, z, cnt = c.join_count(*cols)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        assert np.array_equal(host(cnt), oc.astype(np.int32))
        plan = c.partition(*cols)
        n_x = plan.info["n_x"]
        assert plan.info["n_z_dense"] == plan.info["n_z"]
        parts = [plan.join_project(a, b) for a, b in ((0, 1000), (1000, n_x))]
        plan.close()
        assert np.array_equal(np.concatenate([host(p[0]) for p in parts]), ox)
        assert np.array_equal(np.concatenate([host(p[1]) for p in parts]), oz)
    finally:
        c.close()


@pytest.mark.parametrize("tile_n", [128, 256])
def test_tc_tile_widths_batch(tile_n):
    insts = [gen.small_two_table(60 + i, n_r=4000 + 900 * i, n_s=3000 + 500 * i, nx=150 + 40 * i, ny=90, nz=170 + 30 * i,
                                 zipf=1.0) for i in range(7)]
    c = ctx_with({dim3.OPT_THETA_Z: 3, dim3.OPT_DENSE_VARIANT: dim3.DENSE_TC, dim3.OPT_DENSE_TILE_N: tile_n})
    try:
        x, z, per = c.batch_join_project([inst_dev(i) for i in insts])
        off = np.concatenate([[0], np.cumsum(per)])
        for t, i in enumerate(insts):
            ox, oz, _ = oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)
            assert np.array_equal(host(x[off[t]:off[t + 1]]), ox) and np.array_equal(host(z[off[t]:off[t + 1]]), oz)
    finally:
        c.close()


def test_dense_tile_option_range():
    c = dim3.Context(0)
    try:
        for bad in (64, 192, 512):
            with pytest.raises(dim3.Dim3Error):
                c.set_option(dim3.OPT_DENSE_TILE_N, bad)
    finally:
        c.close()
