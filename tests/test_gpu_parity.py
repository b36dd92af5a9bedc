"""Parity of the CUDA path with the CPU oracle, element by element, on
seeded inputs that span several tiles, ragged tails and the degenerate cases.
All integer work: the bar is bit-exact equality."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import check_sorted_distinct, dev, host, inst_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, dim3.PATH_HYBRID)  # these tests target the hybrid kernels
    yield c
    c.close()


def fresh_ctx(opts):
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, dim3.PATH_HYBRID)
    for k, v in opts.items():
        c.set_option(k, v)
    return c


def project(ctx, inst):
    x, z = ctx.join_project(*inst_dev(inst))
    torch.cuda.synchronize()
    return host(x), host(z)


def count(ctx, inst):
    x, z, c = ctx.join_count(*inst_dev(inst))
    torch.cuda.synchronize()
    return host(x), host(z), host(c)


def assert_project(ctx, inst):
    gx, gz = project(ctx, inst)
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert gx.size == ox.size, f"{inst.name}: {gx.size} pairs vs oracle {ox.size}"
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz)


def assert_count(ctx, inst):
    gx, gz, gc = count(ctx, inst)
    ox, oz, oc, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert gx.size == ox.size
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz) and np.array_equal(gc, oc.astype(np.int32))


# ------------------------------------------------------------------ mapping
@pytest.mark.parametrize("n,pool", [(1, 1), (7, 3), (1000, 10), (100_000, 5000), (1_000_003, 200_000),
                                    (300_000, 300_000)])
def test_map_parity(ctx, n, pool):
    rng = np.random.default_rng(n + pool)
    p = gen.random_ids(rng, pool)
    vals = p[rng.integers(0, pool, size=n)]
    ids, d = ctx.map(dev(vals))
    oids, od = oracle.rank_map(vals)
    assert np.array_equal(host(d), od) and np.array_equal(host(ids), oids)


def test_map_edge_values(ctx):
    vals = np.array([2**31 - 1, -2**31, 0, -1, 1, -2**31, 2**31 - 1, 0], np.int32)
    ids, d = ctx.map(dev(vals))
    oids, od = oracle.rank_map(vals)
    assert np.array_equal(host(d), od) and np.array_equal(host(ids), oids)
    ids, d = ctx.map(dev(np.zeros(0, np.int32)))
    assert ids.numel() == 0 and d.numel() == 0


# ---------------------------------------------------------------- partition
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("theta", [0, 3, 12, 1 << 30])
def test_partition_parity(ctx, seed, theta):
    inst = gen.small_two_table(seed, n_r=5000, n_s=4000, nx=400, ny=300, nz=350, zipf=1.1,
                               dup_frac=0.1 if seed % 2 else 0.0, self_join=(seed == 3))
    plan = ctx.partition(*inst_dev(inst), theta_z=theta)
    o = oracle.plan(inst.r_key, inst.r_val, inst.s_key, inst.s_val, theta)
    info = plan.info
    assert info["n_x"] == o.dict_x.size and info["n_y"] == o.dict_y.size and info["n_z"] == o.dict_z.size
    assert info["out_j"] == o.out_j
    assert info["n_r_kept"] == o.r_col.size
    assert info["n_z_dense"] == int(o.dense_z.sum())
    for name, ref in [("dict_x", o.dict_x), ("dict_y", o.dict_y), ("dict_z", o.dict_z), ("r_rowptr", o.r_rowptr),
                      ("r_col", o.r_col), ("m_z", o.m_z), ("ss_rowptr", o.ss_rowptr), ("ss_col", o.ss_col),
                      ("deg_s", o.deg_s)]:
        got = host(plan.export(name))
        assert np.array_equal(got.astype(np.int64), np.asarray(ref).astype(np.int64)), name
    assert np.array_equal(host(plan.export("dense_z")).astype(bool), o.dense_z)
    outj_x = np.add.reduceat(o.deg_s[o.r_col], o.r_rowptr[:-1]) if o.r_col.size else np.zeros(0)
    outj_x = np.where(np.diff(o.r_rowptr) > 0, outj_x, 0)
    assert np.array_equal(host(plan.export("outj_x")), outj_x.astype(np.int64))
    plan.close()


# ----------------------------------------------------------- join (small)
@pytest.mark.parametrize("seed", range(16))
def test_join_small_random(ctx, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) for v in rng.integers(1, 300, size=3))
    inst = gen.small_two_table(seed, n_r=int(rng.integers(0, 4000)), n_s=int(rng.integers(0, 4000)),
                               nx=nx, ny=ny, nz=nz, zipf=[None, 0.8, 1.2][seed % 3],
                               dup_frac=0.2 if seed % 4 == 1 else 0.0, self_join=(seed % 5 == 0))
    assert_project(ctx, inst)
    assert_count(ctx, inst)


def test_fig3_example(ctx):
    # Section 2.3: (x2, z2) produced by two joins, emitted once; whichever side z2 is on
    r_key, r_val = np.array([1, 3], np.int32), np.array([2, 2], np.int32)
    s_key, s_val = np.array([1, 3], np.int32), np.array([2, 2], np.int32)
    for theta in (0, 1 << 30):
        c = fresh_ctx({dim3.OPT_THETA_Z: theta})
        x, z, cnt = c.join_count(dev(r_key), dev(r_val), dev(s_key), dev(s_val))
        assert host(x).tolist() == [2] and host(z).tolist() == [2] and host(cnt).tolist() == [2]
        c.close()


@pytest.mark.parametrize("case", ["empty_r", "empty_s", "both_empty", "no_overlap", "single"])
def test_degenerate(ctx, case):
    e = np.zeros(0, np.int32)
    one = np.array([5], np.int32)
    args = {
        "empty_r": (e, e, one, one),
        "empty_s": (one, one, e, e),
        "both_empty": (e, e, e, e),
        "no_overlap": (np.array([1, 2], np.int32), np.array([7, 8], np.int32), np.array([3], np.int32), one),
        "single": (one, np.array([9], np.int32), one, np.array([-4], np.int32)),
    }[case]
    inst = gen.Instance(case, *args)
    assert_project(ctx, inst)
    assert_count(ctx, inst)


def test_config1_self_20k(ctx):
    inst = gen.config1_self()
    assert_project(ctx, inst)
    assert_count(ctx, inst)


@pytest.mark.parametrize("scale", [0.01, 0.03])
def test_config2_scaled(ctx, scale):
    inst = gen.config2_two_table(scale=scale)
    assert_project(ctx, inst)


def test_config2_scaled_count(ctx):
    assert_count(ctx, gen.config2_two_table(scale=0.02))


def test_chung_lu_small(ctx):
    inst = gen.chung_lu_self(np.random.default_rng(9), 20_000, 80_000, 2.1)
    assert_project(ctx, inst)
    assert_count(ctx, inst)


@pytest.mark.parametrize("which", ["cfg1", "chung_lu", "dups"])
@pytest.mark.parametrize("theta", [-1, 4])
def test_self_join_shared_pointers(ctx, which, theta):
    """R and S given by the same tensors (the library maps once) and by
    separate copies give the same plan sizes and results, equal to the oracle."""
    if which == "cfg1":
        inst = gen.config1_self()
    elif which == "chung_lu":
        inst = gen.chung_lu_self(np.random.default_rng(11), 5_000, 20_000, 2.1)
    else:
        inst = gen.small_two_table(21, 3000, 3000, 300, 300, 150, dup_frac=0.2, self_join=True)
    assert inst.self_join
    shared = inst_dev(inst)
    assert shared[0].data_ptr() == shared[2].data_ptr()
    separate = inst_dev(inst, share_self=False)
    infos = []
    for cols in (shared, separate):
        plan = ctx.partition(*cols, theta_z=theta)
        try:
            infos.append({k: plan.info[k] for k in ("n_x", "n_y", "n_z", "out_j", "n_z_dense", "n_s_sparse")})
        finally:
            plan.close()
    assert infos[0] == infos[1] and infos[0]["n_x"] == infos[0]["n_z"]
    ox, oz, oc = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[:3]
    for cols in (shared, separate):
        x, z, c = ctx.join_count(*cols)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        assert np.array_equal(host(c), oc.astype(np.int32))
        x, z = ctx.join_project(*cols)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)


# ------------------------------------------- invariance to split and variants
@pytest.mark.parametrize("variant", [dim3.DENSE_TC, dim3.DENSE_POPC, dim3.DENSE_PROBE])
@pytest.mark.parametrize("theta", [0, 5, 40, 1 << 30])
def test_dense_variants_and_threshold(variant, theta):
    """Section 2.3 and 2.6: the result does not depend on the dense/sparse
    threshold or on the bitmap-intersection method."""
    c = fresh_ctx({dim3.OPT_THETA_Z: theta, dim3.OPT_DENSE_VARIANT: variant})
    for seed in range(3):
        inst = gen.small_two_table(100 + seed, n_r=6000, n_s=5000, nx=700, ny=500, nz=600, zipf=1.0,
                                   dup_frac=0.05)
        assert_project(c, inst)
        assert_count(c, inst)
    assert_project(c, gen.config1_self())
    c.close()


@pytest.mark.parametrize("variant", [dim3.DENSE_TC, dim3.DENSE_POPC])
def test_dense_multi_tile(variant):
    """DenseEC over several 128 x 256 tiles and many K blocks with ragged edges."""
    c = fresh_ctx({dim3.OPT_THETA_Z: 0, dim3.OPT_DENSE_VARIANT: variant})
    inst = gen.small_two_table(7, n_r=60_000, n_s=50_000, nx=1000, ny=700, nz=600, zipf=0.9)
    assert_project(c, inst)
    assert_count(c, inst)
    c.close()


@pytest.mark.parametrize("row_min", [0, 1, 1 << 40])
def test_bitmap_rows_invariance(row_min):
    c = fresh_ctx({dim3.OPT_BITMAP_ROW_MIN: row_min})
    inst = gen.config2_two_table(scale=0.01)
    assert_project(c, inst)
    c.close()


# ----------------------------------------------------------- API protocol
def test_capacity_protocol(ctx):
    inst = gen.config1_self()
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    n = ox.size
    out_x = torch.full((n - 1,), -7, dtype=torch.int32, device="cuda")
    out_z = torch.full((n - 1,), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(dim3.Dim3Error) as ei:
        ctx.join_project(*inst_dev(inst), out_x=out_x, out_z=out_z)
    assert ei.value.status == -4
    assert str(n) in str(ei.value)
    # buffer contents after a capacity error are unspecified; writes stayed inside them
    assert out_x.numel() == n - 1
    out_x = torch.empty(n, dtype=torch.int32, device="cuda")
    out_z = torch.empty(n, dtype=torch.int32, device="cuda")
    x, z = ctx.join_project(*inst_dev(inst), out_x=out_x, out_z=out_z)
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)


def test_unaligned_outputs(ctx):
    inst = gen.config2_two_table(scale=0.01)
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    n = ox.size
    bx = torch.empty(n + 3, dtype=torch.int32, device="cuda")
    bz = torch.empty(n + 5, dtype=torch.int32, device="cuda")
    x, z = ctx.join_project(*inst_dev(inst), out_x=bx[1:], out_z=bz[3:])
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)


def test_x_range_chunks(ctx):
    inst = gen.config2_two_table(scale=0.02)
    plan = ctx.partition(*inst_dev(inst))
    nx = plan.info["n_x"]
    cuts = [0, 1, nx // 3, nx // 3, nx - 1, nx]
    xs, zs = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        x, z = plan.join_project(a, b)
        xs.append(host(x))
        zs.append(host(z))
    rc = host(plan.row_counts())
    plan.close()
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert np.array_equal(np.concatenate(xs), ox) and np.array_equal(np.concatenate(zs), oz)
    assert rc.sum() == ox.size
    assert np.array_equal(rc, np.bincount(np.searchsorted(np.unique(ox), ox)))


def test_bad_range_rejected(ctx):
    inst = gen.config1_self()
    plan = ctx.partition(*inst_dev(inst))
    with pytest.raises(dim3.Dim3Error):
        plan.join_project(5, 3)
    with pytest.raises(dim3.Dim3Error):
        plan.join_project(0, plan.info["n_x"] + 1)
    plan.close()


def test_deterministic_repeat(ctx):
    inst = gen.config2_two_table(scale=0.02)
    a = project(ctx, inst)
    b = project(ctx, inst)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_sorted_distinct_on_device(ctx):
    inst = gen.config2_two_table(scale=0.05)
    x, z = ctx.join_project(*inst_dev(inst))
    check_sorted_distinct(x, z)


@pytest.mark.parametrize("rows", [1, 2, 4])
def test_emit_rows_per_cta(rows):
    """The emitting pass gives the same pairs with 1, 2 or 4 x rows per CTA,
    including an odd number of rows (ragged last group)."""
    c = fresh_ctx({6: rows})
    for inst in (gen.config2_two_table(scale=0.01), gen.small_two_table(3, n_r=3001, n_s=2999, nx=301, ny=97,
                                                                          nz=203, zipf=1.1)):
        assert_project(c, inst)
    c.close()


@pytest.mark.parametrize("two_pass", [0, 1])
def test_single_and_two_pass_agree(two_pass):
    """The single-pass emission (decoupled look-back) and the counting +
    emitting passes give the same pairs, for one and two rows per CTA."""
    for rows in (1, 2):
        c = fresh_ctx({7: two_pass, 6: rows})
        for inst in (gen.config2_two_table(scale=0.02), gen.small_two_table(9, n_r=5000, n_s=4000, nx=801, ny=200,
                                                                              nz=300, zipf=1.0)):
            ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
            bx = torch.empty(ox.size + 7, dtype=torch.int32, device="cuda")
            bz = torch.empty(ox.size + 7, dtype=torch.int32, device="cuda")
            x, z = c.join_project(*inst_dev(inst), out_x=bx[1:], out_z=bz[2:])
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        c.close()


def test_single_pass_capacity_short_reports_count():
    inst = gen.config2_two_table(scale=0.01)
    ox, _, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    c = fresh_ctx({})
    bx = torch.empty(ox.size // 2, dtype=torch.int32, device="cuda")
    bz = torch.empty(ox.size // 2, dtype=torch.int32, device="cuda")
    with pytest.raises(dim3.Dim3Error) as ei:
        c.join_project(*inst_dev(inst), out_x=bx, out_z=bz)
    assert ei.value.status == -4 and str(ox.size) in str(ei.value)
    c.close()


@pytest.fixture(scope="module")
def density_mix():
    """A dense-output (99 %), a mixed (37 %), a 3 % and a 1 % output density
    instance with their oracle results."""
    insts = (gen.small_two_table(11, n_r=20_000, n_s=20_000, nx=400, ny=50, nz=3000, zipf=0.9),
             gen.small_two_table(12, n_r=30_000, n_s=30_000, nx=2000, ny=3000, nz=40_000, zipf=1.1),
             gen.chung_lu_self(np.random.default_rng(13), 20_000, 80_000, 2.1),
             gen.chung_lu_self(np.random.default_rng(13), 60_000, 120_000, 2.1))
    return [(inst, *oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[:2]) for inst in insts]


@pytest.mark.parametrize("id_max", [0, 64, 512, 1024])
def test_id_chunk_threshold(id_max, density_mix):
    """Every split between staged-id chunks and group-by-group compaction,
    with one x row per CTA (the kernel whose stage size follows the output
    density), single pass and two passes."""
    for two_pass in (0, 1):
        c = fresh_ctx({6: 1, 7: two_pass, 8: id_max})
        for inst, ox, oz in density_mix:
            bx = torch.empty(ox.size + 4, dtype=torch.int32, device="cuda")
            bz = torch.empty(ox.size + 4, dtype=torch.int32, device="cuda")
            x, z = c.join_project(*inst_dev(inst), out_x=bx, out_z=bz)
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), inst.name
        c.close()


def test_id_chunk_threshold_range():
    c = fresh_ctx({})
    with pytest.raises(dim3.Dim3Error):
        c.set_option(8, 1025)
    c.close()


def _wide_sparse(seed, n, ny):
    rng = np.random.default_rng(seed)
    return gen.Instance("wide_sparse", rng.integers(0, ny, n).astype(np.int32),
                        rng.integers(-10**7, 10**7, n).astype(np.int32), rng.integers(0, ny, n).astype(np.int32),
                        rng.integers(-10**7, 10**7, n).astype(np.int32))


@pytest.fixture(scope="module")
def wide_insts():
    insts = (_wide_sparse(71, 200_000, 50_000), gen.chung_lu_self(np.random.default_rng(72), 100_000, 200_000, 2.1))
    return [(inst, *oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[:2]) for inst in insts]


@pytest.mark.parametrize("light_max", [-1, 0, 5, 1024])
def test_light_rows(light_max, wide_insts):
    """Rows with few join tuples on a wide z range are deduplicated by sorting
    (any threshold gives the SPA's result): uniform sparse tables, a power-law
    graph with hubs (heavy rows) among light rows, both passes and x ranges."""
    c = fresh_ctx({4: light_max})
    for inst, ox, oz in wide_insts:
        gx, gz = project(c, inst)
        assert np.array_equal(gx, ox) and np.array_equal(gz, oz), inst.name
        plan = c.partition(*inst_dev(inst))
        n_x = plan.info["n_x"]
        xs, zs = [], []
        for a, b in ((0, n_x // 2), (n_x // 2, n_x)):
            x, z = plan.join_project(a, b)
            xs.append(host(x))
            zs.append(host(z))
        plan.close()
        assert np.array_equal(np.concatenate(xs), ox) and np.array_equal(np.concatenate(zs), oz)
    c.close()
