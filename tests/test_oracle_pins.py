"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these tests re-types the oracle's own algorithm: each pin comes from
somewhere else (brute force over all (x, z) pairs, a library boolean matrix
product, the paper's textual examples, closed forms, invariants), chosen so
that a dropped term, a wrong index, a swapped operand or a missed dedup in the
oracle fails at least one of them.
"""

import itertools
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_force(r_key, r_val, s_key, s_val):
    """Eq. 1 by exhaustion: every (x, z) in X x Z with at least one common y;
    the count is the number of such y (Section 4.1 with COUNT)."""
    R = set(zip(map(int, r_val), map(int, r_key)))
    S = set(zip(map(int, s_val), map(int, s_key)))
    X = sorted({x for x, _ in R})
    Z = sorted({z for z, _ in S})
    Y = sorted({y for _, y in R} | {y for _, y in S})
    out = []
    for x in X:
        for z in Z:
            c = sum(1 for y in Y if (x, y) in R and (z, y) in S)
            if c:
                out.append((x, z, c))
    return out


def as_triples(x, z, c):
    return list(zip(map(int, x), map(int, z), map(int, c)))


def tiny(seed, **kw):
    return gen.small_two_table(seed, **kw)


@pytest.mark.parametrize("seed", range(24))
def test_bruteforce_tiny(seed):
    rng = np.random.default_rng(1000 + seed)
    nx, ny, nz = (int(v) for v in rng.integers(1, 12, size=3))
    inst = tiny(seed, n_r=int(rng.integers(0, 40)), n_s=int(rng.integers(0, 40)),
                nx=nx, ny=ny, nz=nz, dup_frac=0.3 if seed % 2 else 0.0,
                self_join=(seed % 5 == 0))
    x, z, c, out_j = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert as_triples(x, z, c) == brute_force(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    px, pz, pj = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert np.array_equal(px, x) and np.array_equal(pz, z) and pj == out_j


@pytest.mark.parametrize("seed", range(6))
def test_boolean_matmul(seed):
    """Section 1.1, MM formulation: C = R S over 0/1 matrices, (x, z) is in
    the result iff C[x, z] > 0, and C[x, z] is the COUNT."""
    inst = tiny(seed, n_r=300, n_s=250, nx=30, ny=20, nz=25, zipf=1.0)
    X = np.unique(inst.r_val)
    Y = np.unique(np.concatenate([inst.r_key, inst.s_key]))
    Z = np.unique(inst.s_val)
    Rm = np.zeros((X.size, Y.size), np.int64)
    Sm = np.zeros((Y.size, Z.size), np.int64)
    Rm[np.searchsorted(X, inst.r_val), np.searchsorted(Y, inst.r_key)] = 1
    Sm[np.searchsorted(Y, inst.s_key), np.searchsorted(Z, inst.s_val)] = 1
    C = Rm @ Sm
    ii, jj = np.nonzero(C)  # row-major order = canonical order (X, Z sorted)
    x, z, c, out_j = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert np.array_equal(x, X[ii]) and np.array_equal(z, Z[jj])
    assert np.array_equal(c, C[ii, jj])
    assert out_j == int(C.sum())


def _read_golden(name):
    rows = {"R": [], "S": [], "PAIR": [], "DROP": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                rows[line[0]].append([int(v) for v in line[1:]])
    return rows


def test_fig3_single_emission():
    """Section 2.3: (x2, z2) is produced by two joins but appears once."""
    g = _read_golden("fig3_intersection_free.txt")
    R = np.array(g["R"], np.int32)
    S = np.array(g["S"], np.int32)
    x, z, c, out_j = oracle.join_count(R[:, 1], R[:, 0], S[:, 1], S[:, 0])
    assert as_triples(x, z, c) == [tuple(p) for p in g["PAIR"]]
    assert out_j == 2  # two join tuples, one projected pair


def test_fig2_semijoin_reconstruction():
    """Section 2.2, Optimization 2: R tuples whose y is not in S.y are dropped
    and contribute nothing (reconstructed example)."""
    g = _read_golden("fig2_semijoin.txt")
    R = np.array(g["R"], np.int32)
    S = np.array(g["S"], np.int32)
    p = oracle.plan(R[:, 1], R[:, 0], S[:, 1], S[:, 0], theta_z=1 << 30)
    assert sorted(np.nonzero(~p.r_keep)[0].tolist()) == [d[0] for d in g["DROP"]]
    x, z, c, _ = oracle.join_count(R[:, 1], R[:, 0], S[:, 1], S[:, 0])
    assert as_triples(x, z, c) == [tuple(q) for q in g["PAIR"]]
    keep = p.r_keep
    x2, z2, c2, _ = oracle.join_count(R[keep, 1], R[keep, 0], S[:, 1], S[:, 0])
    assert as_triples(x2, z2, c2) == as_triples(x, z, c)


@pytest.mark.parametrize("nx,ny,nz", [(1, 1, 1), (7, 5, 3), (40, 30, 20)])
def test_full_matrices(nx, ny, nz):
    """Section 2.7, special case alpha = beta = 1: OUT_P = |X||Z|, every count
    is |Y|, |OUT_J| = |X||Y||Z|."""
    rng = np.random.default_rng(nx * 100 + ny)
    X, Y, Z = gen.random_ids(rng, nx), gen.random_ids(rng, ny), gen.random_ids(rng, nz)
    rx, ry = (a.ravel() for a in np.meshgrid(X, Y, indexing="ij"))
    sz, sy = (a.ravel() for a in np.meshgrid(Z, Y, indexing="ij"))
    perm = rng.permutation(rx.size)
    x, z, c, out_j = oracle.join_count(ry[perm], rx[perm], sy, sz)
    assert x.size == nx * nz
    assert np.all(c == ny)
    assert out_j == nx * ny * nz
    exp = sorted(itertools.product(sorted(X.tolist()), sorted(Z.tolist())))
    assert list(zip(x.tolist(), z.tolist())) == exp


@pytest.mark.parametrize("seed", range(8))
def test_out_j_closed_form(seed):
    """|OUT_J| = sum over y of deg_R(y) * deg_S(y) (distinct tuples); the
    counts sum to |OUT_J|; OUT_P <= OUT_J."""
    inst = tiny(seed, n_r=2000, n_s=1500, nx=80, ny=60, nz=70, zipf=1.1, dup_frac=0.2)
    x, z, c, out_j = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    ru = np.unique(np.stack([inst.r_val, inst.r_key], 1), axis=0)
    su = np.unique(np.stack([inst.s_val, inst.s_key], 1), axis=0)
    yr, cr = np.unique(ru[:, 1], return_counts=True)
    ys, cs = np.unique(su[:, 1], return_counts=True)
    common, ir, is_ = np.intersect1d(yr, ys, return_indices=True)
    closed = int((cr[ir].astype(np.int64) * cs[is_]).sum())
    assert out_j == closed == int(c.sum())
    assert x.size <= out_j


def test_matching_no_duplicates():
    """When every (x, z) shares at most one y, nothing is deduplicated:
    OUT_P = OUT_J and every count is 1."""
    rng = np.random.default_rng(7)
    n = 500
    X, Y, Z = gen.random_ids(rng, n), gen.random_ids(rng, n), gen.random_ids(rng, n)
    # R: x_i - y_i (a matching); S: each y_j joined to two z's, z_j and z_{j+1}
    r_key, r_val = Y, X
    s_key = np.concatenate([Y, Y])
    s_val = np.concatenate([Z, np.roll(Z, 1)])
    x, z, c, out_j = oracle.join_count(r_key, r_val, s_key, s_val)
    assert x.size == out_j == 2 * n
    assert np.all(c == 1)


@pytest.mark.parametrize("seed", range(4))
def test_shuffle_and_duplicate_invariance(seed):
    """Inputs are sets in arbitrary order (the paper shuffles them): row order
    and repeated rows must not change the result."""
    inst = tiny(seed, n_r=800, n_s=700, nx=50, ny=40, nz=45, zipf=1.0)
    base = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    rng = np.random.default_rng(seed)
    pr = rng.permutation(inst.nr)
    ps = rng.permutation(inst.ns)
    rr = np.concatenate([pr, pr[: inst.nr // 3]])
    ss = np.concatenate([ps, ps[: inst.ns // 2]])
    other = oracle.join_count(inst.r_key[rr], inst.r_val[rr], inst.s_key[ss], inst.s_val[ss])
    for a, b in zip(base, other):
        assert np.array_equal(a, b)


def test_canonical_signed_order():
    """Canonical order compares signed int32: negative ids first."""
    r_val = np.array([5, -3, 2147483647, -2147483648], np.int32)
    r_key = np.array([1, 1, 1, 1], np.int32)
    s_val = np.array([-1, 0, 7], np.int32)
    s_key = np.array([1, 1, 1], np.int32)
    x, z, _ = oracle.join_project(r_key, r_val, s_key, s_val)
    pairs = list(zip(x.tolist(), z.tolist()))
    assert pairs == sorted(pairs)
    assert pairs[0] == (-2147483648, -1) and pairs[-1] == (2147483647, 7)


def test_monotone_relabel():
    """Relabelling every column by a strictly increasing map relabels the
    output element-wise and keeps its order."""
    inst = tiny(3, n_r=600, n_s=600, nx=40, ny=30, nz=35, zipf=0.9)
    x, z, c, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)

    vals = np.unique(np.concatenate([inst.r_val, inst.s_val, inst.r_key, inst.s_key]))
    new_vals = np.sort(gen.random_ids(np.random.default_rng(5), vals.size))

    def f(v):  # strictly increasing on the values that occur
        return new_vals[np.searchsorted(vals, v)]

    x2, z2, c2, _ = oracle.join_count(f(inst.r_key), f(inst.r_val), f(inst.s_key), f(inst.s_val))
    assert np.array_equal(x2, f(x)) and np.array_equal(z2, f(z)) and np.array_equal(c2, c)


@pytest.mark.parametrize("seed", range(5))
def test_rank_map_against_unique(seed):
    """Order-preserving mapping equals numpy's sort-based unique inverse."""
    rng = np.random.default_rng(seed)
    pool = gen.random_ids(rng, 1 + seed * 97)
    vals = pool[rng.integers(0, pool.size, size=3000)]
    ids, d = oracle.rank_map(vals)
    u, inv = np.unique(vals, return_inverse=True)
    assert np.array_equal(d, u) and np.array_equal(ids, inv)
    assert np.array_equal(d[ids], vals)
    assert np.all(np.diff(d.astype(np.int64)) > 0)


def test_rank_map_empty_and_single():
    ids, d = oracle.rank_map(np.zeros(0, np.int32))
    assert ids.size == 0 and d.size == 0
    ids, d = oracle.rank_map(np.array([-5, -5, -5], np.int32))
    assert ids.tolist() == [0, 0, 0] and d.tolist() == [-5]


@pytest.mark.parametrize("seed", range(6))
def test_intersection_free_split(seed):
    """Section 2.3: splitting S by z makes the dense and sparse results
    disjoint, with union equal to the full result, for any threshold."""
    inst = tiny(seed, n_r=1500, n_s=1200, nx=60, ny=40, nz=50, zipf=1.2)
    full = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    full_set = set(as_triples(*full[:3]))
    zs, mz = np.unique(np.unique(np.stack([inst.s_val, inst.s_key], 1), axis=0)[:, 0],
                       return_counts=True)
    for theta in [0, 1, int(np.median(mz)), int(mz.max()), int(mz.max()) + 1]:
        dense_z = set(zs[mz >= theta].tolist())
        dm = np.isin(inst.s_val, list(dense_z)) if dense_z else np.zeros(inst.ns, bool)
        d = oracle.join_count(inst.r_key, inst.r_val, inst.s_key[dm], inst.s_val[dm])
        s = oracle.join_count(inst.r_key, inst.r_val, inst.s_key[~dm], inst.s_val[~dm])
        dset, sset = set(as_triples(*d[:3])), set(as_triples(*s[:3]))
        assert not (dset & sset)
        assert dset | sset == full_set
        assert d[3] + s[3] == full[3]


def test_x_filter_rows():
    """Restricting R to some x gives exactly those rows of the full result."""
    inst = tiny(11, n_r=3000, n_s=2500, nx=100, ny=50, nz=80, zipf=1.0)
    x, z, c, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    pick = np.unique(inst.r_val)[::7]
    xf, zf, cf, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val, x_filter=pick)
    m = np.isin(x, pick)
    assert np.array_equal(xf, x[m]) and np.array_equal(zf, z[m]) and np.array_equal(cf, c[m])


@pytest.mark.parametrize("seed", range(6))
def test_plan_definitions(seed):
    """Mapping/partition quantities against plain Python sets and counters."""
    inst = tiny(seed, n_r=300, n_s=260, nx=20, ny=15, nz=18, zipf=1.0, dup_frac=0.2)
    theta = 3 + seed
    p = oracle.plan(inst.r_key, inst.r_val, inst.s_key, inst.s_val, theta)
    S = set(zip(inst.s_val.tolist(), inst.s_key.tolist()))
    sy = {y for _, y in S}
    keep = [int(y) in sy for y in inst.r_key.tolist()]
    assert p.r_keep.tolist() == keep
    R = {(x, y) for (x, y), k in zip(zip(inst.r_val.tolist(), inst.r_key.tolist()), keep) if k}
    assert p.dict_y.tolist() == sorted(sy)
    assert p.dict_x.tolist() == sorted({x for x, _ in R})
    assert p.dict_z.tolist() == sorted({z for z, _ in S})
    for i, x in enumerate(p.dict_x.tolist()):
        ys = sorted(p.dict_y.tolist().index(y) for (xx, y) in R if xx == x)
        assert p.m_x[i] == len(ys)
        assert p.r_col[p.r_rowptr[i]:p.r_rowptr[i + 1]].tolist() == ys
    for i, z in enumerate(p.dict_z.tolist()):
        m = sum(1 for (zz, _) in S if zz == z)
        assert p.m_z[i] == m and bool(p.dense_z[i]) == (m >= theta)
    outj = 0
    for j, y in enumerate(p.dict_y.tolist()):
        dr = sum(1 for (_, yy) in R if yy == y)
        ds = sum(1 for (_, yy) in S if yy == y)
        assert p.deg_r[j] == dr and p.deg_s[j] == ds
        outj += dr * ds
        sparse_z = sorted(p.dict_z.tolist().index(z) for (z, yy) in S
                          if yy == y and not p.dense_z[p.dict_z.tolist().index(z)])
        assert p.ss_col[p.ss_rowptr[j]:p.ss_rowptr[j + 1]].tolist() == sparse_z
    assert p.out_j == outj
    assert p.out_j == oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)[2]


def test_empty_inputs():
    e = np.zeros(0, np.int32)
    one = np.array([1], np.int32)
    for args in [(e, e, e, e), (one, one, e, e), (e, e, one, one)]:
        x, z, c, j = oracle.join_count(*args)
        assert x.size == 0 and j == 0
    # no common y
    x, z, c, j = oracle.join_count(np.array([1], np.int32), one, np.array([2], np.int32), one)
    assert x.size == 0 and j == 0


def test_config1_sizes():
    """The 20K self-join workload: sizes stated in the input recipe."""
    inst = gen.config1_self()
    assert inst.nr == 20000 and np.unique(inst.r_val).size == 2000
    x, z, c, out_j = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    # self join: symmetric result, full diagonal
    pairs = set(zip(x.tolist(), z.tolist()))
    assert all((b, a) in pairs for a, b in list(pairs)[:2000])
    assert all((v, v) in pairs for v in np.unique(inst.r_val).tolist())
    assert out_j == int(c.sum())
