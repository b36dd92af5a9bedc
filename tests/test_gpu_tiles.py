"""SparseBMM over z ranges wider than one shared-memory bitmap: one CTA per
x row sweeps the z tiles; the counting pass stages every row's z values and
the emitting pass places them (without staging -- DIM3_OPT_TWO_PASS, or
after a plain row count -- the emitting pass rebuilds the tiles). Small
tiles are forced with DIM3_OPT_TILE_WORDS so that inputs the oracle finishes
in seconds span many tiles, with ragged last tiles and tile sizes that are
not whole 1024-z groups; the full-size power-law workload (three tiles of the
default size) is covered in test_gpu_full.py. All integer: exact equality
with the oracle."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import host, inst_dev

pytestmark = pytest.mark.gpu


def _uniform_wide(seed, n, ny, zrange):
    rng = np.random.default_rng(seed)
    return gen.Instance("uniform_wide", rng.integers(0, ny, n).astype(np.int32),
                        rng.integers(-zrange, zrange, n).astype(np.int32), rng.integers(0, ny, n).astype(np.int32),
                        rng.integers(-zrange, zrange, n).astype(np.int32))


@pytest.fixture(scope="module")
def cases():
    insts = (gen.chung_lu_self(np.random.default_rng(81), 120_000, 300_000, 2.1),
             _uniform_wide(82, 300_000, 20_000, 10**8),
             gen.small_two_table(83, n_r=150_000, n_s=150_000, nx=20_000, ny=8_000, nz=200_000, zipf=1.0))
    return [(inst, *oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[:2]) for inst in insts]


def ctx_with(opts):
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, dim3.PATH_HYBRID)
    for k, v in opts.items():
        c.set_option(k, v)
    return c


@pytest.mark.parametrize("light", [-1, 0])
@pytest.mark.parametrize("tile_words", [1024, 1500, 4096])
def test_tiles_vs_oracle(tile_words, light, cases):
    """One call into caller buffers at unaligned offsets, and the plan path
    over two x ranges, with and without the light-row kernel beside the
    tiles."""
    c = ctx_with({dim3.OPT_TILE_WORDS: tile_words, dim3.OPT_LIGHT_ROW_MAX: light})
    try:
        for inst, ox, oz in cases:
            cols = inst_dev(inst)
            bx = torch.empty(ox.size + 5, dtype=torch.int32, device="cuda")
            bz = torch.empty(ox.size + 5, dtype=torch.int32, device="cuda")
            x, z = c.join_project(*cols, out_x=bx[1:], out_z=bz[3:])
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), inst.name
            plan = c.partition(*cols)
            n_x = plan.info["n_x"]
            rc = host(plan.row_counts())
            assert rc.sum() == ox.size
            parts = [plan.join_project(a, b) for a, b in ((0, n_x // 3), (n_x // 3, n_x))]
            plan.close()
            assert np.array_equal(np.concatenate([host(p[0]) for p in parts]), ox)
            assert np.array_equal(np.concatenate([host(p[1]) for p in parts]), oz)
    finally:
        c.close()


@pytest.mark.parametrize("variant", [dim3.DENSE_TC, dim3.DENSE_POPC])
def test_tiles_with_wide_rows_and_dense_part(variant, cases):
    """Wide S_sparse rows (held as z-bitmaps, OR-ed per tile) and DenseEC
    results over the dense z index, both inside the tiled units."""
    c = ctx_with({dim3.OPT_TILE_WORDS: 1024, dim3.OPT_BITMAP_ROW_MIN: 24, dim3.OPT_THETA_Z: 12,
                  dim3.OPT_DENSE_VARIANT: variant})
    try:
        for inst, ox, oz in cases:
            x, z = c.join_project(*inst_dev(inst))
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), inst.name
    finally:
        c.close()


def test_tile_option_range():
    c = dim3.Context(0)
    try:
        for bad in (1, 1023, 12289):
            with pytest.raises(dim3.Dim3Error):
                c.set_option(dim3.OPT_TILE_WORDS, bad)
        c.set_option(dim3.OPT_TILE_WORDS, 0)
    finally:
        c.close()


@pytest.mark.parametrize("light", [-1, 0, 64])
def test_tiles_plan_range_row_counts_and_capacity(light, cases):
    """Tiled rows on a plan x range into caller buffers: exact pairs, the row
    counts the plan keeps for later queries, and a short buffer reported with
    the exact size."""
    c = ctx_with({dim3.OPT_TILE_WORDS: 1024, dim3.OPT_LIGHT_ROW_MAX: light})
    try:
        for inst, ox, oz in cases:
            cols = inst_dev(inst)
            plan = c.partition(*cols)
            n_x = plan.info["n_x"]
            a, b = n_x // 5, n_x - n_x // 7
            dx = host(plan.export("dict_x"))
            sel = (ox >= dx[a]) & (ox <= dx[b - 1])
            bx = torch.empty(int(sel.sum()) + 2, dtype=torch.int32, device="cuda")
            bz = torch.empty(int(sel.sum()) + 2, dtype=torch.int32, device="cuda")
            x, z = plan.join_project(a, b, out_x=bx[1:], out_z=bz[1:])
            assert np.array_equal(host(x), ox[sel]) and np.array_equal(host(z), oz[sel]), inst.name
            ux, cnt = np.unique(ox[sel], return_counts=True)
            exp = np.zeros(b - a, np.int64)
            exp[np.searchsorted(dx[a:b], ux)] = cnt
            assert np.array_equal(host(plan.row_counts(a, b)), exp), inst.name
            plan.close()
            short = torch.empty(ox.size // 2 + 1, dtype=torch.int32, device="cuda")
            with pytest.raises(dim3.Dim3Error) as ei:
                c.join_project(*cols, out_x=short, out_z=short.clone())
            assert ei.value.status == dim3.DIM3_ERR_CAPACITY and str(ox.size) in str(ei.value)
    finally:
        c.close()


@pytest.mark.parametrize("light", [-1, 0, 200])
def test_light_and_bitmap_rows_on_tiles(light, cases):
    """Light rows (warp sorts) beside bitmap rows swept over z tiles, on tiled
    and untiled z ranges, one call and plan x ranges."""
    for tw in (0, 1024):
        c = ctx_with({dim3.OPT_LIGHT_ROW_MAX: light, dim3.OPT_TILE_WORDS: tw})
        try:
            for inst, ox, oz in cases:
                x, z = c.join_project(*inst_dev(inst))
                assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), (inst.name, tw)
                plan = c.partition(*inst_dev(inst))
                n_x = plan.info["n_x"]
                parts = [plan.join_project(a, b) for a, b in ((0, n_x // 2), (n_x // 2, n_x))]
                plan.close()
                assert np.array_equal(np.concatenate([host(p[0]) for p in parts]), ox)
                assert np.array_equal(np.concatenate([host(p[1]) for p in parts]), oz)
        finally:
            c.close()


@pytest.mark.parametrize("two_pass", [0, 1])
@pytest.mark.parametrize("light", [-1, 0])
def test_staged_and_rebuilt_emission_agree(two_pass, light, cases):
    """One call with the rows' z values staged by the counting pass (default)
    or rebuilt by the emitting pass (DIM3_OPT_TWO_PASS), into aligned and
    4-byte-offset output buffers: the same exact pairs."""
    c = ctx_with({dim3.OPT_TILE_WORDS: 1500, dim3.OPT_LIGHT_ROW_MAX: light, dim3.OPT_TWO_PASS: two_pass})
    try:
        for inst, ox, oz in cases:
            cols = inst_dev(inst)
            for shift in (0, 1):
                bx = torch.empty(ox.size + shift, dtype=torch.int32, device="cuda")
                bz = torch.empty(ox.size + shift, dtype=torch.int32, device="cuda")
                x, z = c.join_project(*cols, out_x=bx[shift:], out_z=bz[shift:])
                assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), (inst.name, shift)
    finally:
        c.close()
