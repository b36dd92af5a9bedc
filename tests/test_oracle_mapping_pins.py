"""Pins of the Section 2.2 mapping variants in the oracle (``oracle/mapping.py``).

Each pin comes from outside the oracle's own code path: brute force over
Python tuples and integers, numpy's ``unique`` on 64-bit integers (an int64
key is the pair (high word signed, low word unsigned)), the worked example of
Section 2.2 (a two-attribute join key, projections that include the join key)
computed by nested loops, and the invariance of Eq. 1 under any renaming of
values by a bijection. ``test_mutation_*`` plant plausible mistakes in a copy
of the oracle and check that a pin fails.
"""

import itertools

import numpy as np
import pytest

import oracle
import oracle.mapping as om
from tests.test_oracle_pins import brute_force


def brute_map(rows):
    """Ranks of Python tuples (Python integer order, lexicographic) and the
    first row of each distinct tuple."""
    distinct = sorted(set(rows))
    pos = {t: i for i, t in enumerate(distinct)}
    ids = [pos[t] for t in rows]
    first = [min(i for i, t in enumerate(rows) if t == d) for d in distinct]
    return ids, first


@pytest.mark.parametrize("seed", range(12))
def test_map_tuples_bruteforce_signed(seed):
    rng = np.random.default_rng(seed)
    k = 1 + seed % 3
    n = int(rng.integers(0, 40))
    cols = [rng.integers(-3, 4, n).astype(np.int32) for _ in range(k)]
    ids, first, d = oracle.map_tuples(cols)
    rows = [tuple(int(c[i]) for c in cols) for i in range(n)]
    bids, bfirst = brute_map(rows)
    assert d == len(bfirst)
    assert ids.tolist() == bids and first.tolist() == bfirst


@pytest.mark.parametrize("seed", range(6))
def test_map_tuples_int64_as_words(seed):
    """An int64 column given as (high word signed, low word unsigned) ranks
    exactly like the int64 values themselves (numpy unique)."""
    rng = np.random.default_rng(100 + seed)
    pool = rng.integers(-2**62, 2**62, 50, dtype=np.int64)
    pool[:6] = [0, -1, 1, 2**32 - 1, 2**32, -2**32]  # low words 0, 0xffffffff, carries
    v = rng.choice(pool, 300)
    hi = (v >> 32).astype(np.int32)
    lo = (v & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    ids, first, d = oracle.map_tuples([hi, lo], unsigned_mask=0b10)
    uniq, inv = np.unique(v, return_inverse=True)
    assert d == uniq.size and np.array_equal(ids, inv.astype(np.int32))
    assert np.array_equal(v[first], uniq)
    # the first row of each value: brute force
    assert first.tolist() == [int(np.flatnonzero(v == u)[0]) for u in uniq]


def test_map_tuples_unsigned_single_column():
    v = np.array([-1, 0, 5, -2**31, 2**31 - 1, 0, -1], np.int32)
    ids, _, _ = oracle.map_tuples([v], unsigned_mask=1)
    as_unsigned = [int(x) % 2**32 for x in v]  # two's complement read as unsigned
    bids, _ = brute_map([(u,) for u in as_unsigned])
    assert ids.tolist() == bids


def composite_bruteforce(R, S):
    """Section 2.2's example Pi_{a,b,c,d,e}(R(a,b,c,d) join_{c,d} S(c,d,e,f)) by
    nested loops, as a sorted list of distinct (a, b, c, d, e)."""
    out = set()
    for (a, b, c, d) in R:
        for (c2, d2, e, f) in S:
            if (c, d) == (c2, d2):
                out.add((a, b, c, d, e))
    return sorted(out)


def composite_via_ids(R, S):
    """The same query through the mapping of Section 2.2: x = (a, b),
    y = (c, d), z = (c, d, e), then Pi_{x,z}(R(x,y) join_y S(z,y)) on ids."""
    R = np.asarray(R, np.int32).reshape(-1, 4)
    S = np.asarray(S, np.int32).reshape(-1, 4)
    nr = R.shape[0]
    xid, xfirst, _ = oracle.map_tuples([R[:, 0], R[:, 1]])
    yid, _, _ = oracle.map_tuples([np.concatenate([R[:, 2], S[:, 0]]), np.concatenate([R[:, 3], S[:, 1]])])
    zid, zfirst, _ = oracle.map_tuples([S[:, 0], S[:, 1], S[:, 2]])
    x, z, _ = oracle.join_project_ids(yid[:nr], xid, yid[nr:], zid)
    rows = []
    for xi, zi in zip(x.tolist(), z.tolist()):
        ra, sa = R[xfirst[xi]], S[zfirst[zi]]
        rows.append((int(ra[0]), int(ra[1]), int(sa[0]), int(sa[1]), int(sa[2])))
    return rows


@pytest.mark.parametrize("seed", range(10))
def test_composite_example(seed):
    rng = np.random.default_rng(200 + seed)
    R = [tuple(int(v) for v in rng.integers(-2, 3, 4)) for _ in range(int(rng.integers(0, 30)))]
    S = [tuple(int(v) for v in rng.integers(-2, 3, 4)) for _ in range(int(rng.integers(0, 30)))]
    # canonical order of the id join = lexicographic order of the projected tuples
    assert composite_via_ids(R, S) == composite_bruteforce(R, S)


@pytest.mark.parametrize("seed", range(8))
def test_join_ids_bijection_invariance(seed):
    """Eq. 1 commutes with renaming values by order-preserving bijections: the
    id join, translated back, is the value join (by brute force)."""
    rng = np.random.default_rng(300 + seed)
    nr, ns = int(rng.integers(0, 60)), int(rng.integers(0, 60))
    r_y, r_x = rng.integers(-50, 50, nr), rng.integers(-1000, 1000, nr)
    s_y, s_z = rng.integers(-50, 50, ns), rng.integers(-9, 9, ns)
    ys = sorted(set(r_y.tolist()) | set(s_y.tolist()))
    xs, zs = sorted(set(r_x.tolist())), sorted(set(s_z.tolist()))
    yi = {v: i for i, v in enumerate(ys)}
    xi = {v: i for i, v in enumerate(xs)}
    zi = {v: i for i, v in enumerate(zs)}
    ids = [np.array([m[v] for v in col.tolist()], np.int32)
           for m, col in ((yi, r_y), (xi, r_x), (yi, s_y), (zi, s_z))]
    x, z, c, _ = oracle.join_count_ids(*ids)
    got = [(xs[a], zs[b], int(k)) for a, b, k in zip(x.tolist(), z.tolist(), c.tolist())]
    assert got == brute_force(r_y, r_x, s_y, s_z)
    px, pz, _ = oracle.join_project_ids(*ids)
    assert np.array_equal(px, x) and np.array_equal(pz, z)


@pytest.mark.parametrize("seed", range(6))
def test_join_ids_negative_tuples_dropped(seed):
    """Tuples carrying a negative id are not part of the input: adding them
    changes nothing; an R tuple whose y no S tuple holds adds no pair."""
    rng = np.random.default_rng(400 + seed)
    n = 40
    r_y, r_x = rng.integers(0, 8, n), rng.integers(0, 12, n)
    s_y, s_z = rng.integers(0, 8, n), rng.integers(0, 10, n)
    base = brute_force(r_y, r_x, s_y, s_z)
    junk = rng.integers(0, 8, 15)
    neg = -rng.integers(1, 5, 15)
    r_y2 = np.concatenate([r_y, neg, junk])
    r_x2 = np.concatenate([r_x, junk, neg])
    s_y2 = np.concatenate([s_y, neg, junk, [100] * 3])  # y = 100 never in R
    s_z2 = np.concatenate([s_z, junk, neg, [1, 2, 3]])
    r_y3 = np.concatenate([r_y2, [200, 201]])  # y never in S
    r_x3 = np.concatenate([r_x2, [0, 1]])
    x, z, c, _ = oracle.join_count_ids(r_y3, r_x3, s_y2, s_z2)
    assert list(zip(x.tolist(), z.tolist(), c.tolist())) == base


# ---------------------------------------------------------------- mutations
def _all_pins():
    for s in range(12):
        test_map_tuples_bruteforce_signed(s)
    for s in range(6):
        test_map_tuples_int64_as_words(s)
    test_map_tuples_unsigned_single_column()
    for s in range(10):
        test_composite_example(s)
    for s in range(8):
        test_join_ids_bijection_invariance(s)
    for s in range(6):
        test_join_ids_negative_tuples_dropped(s)


def _unstable_order(cols, unsigned_mask=0):
    ids, first, d = _real_map_tuples(cols, unsigned_mask)
    # plausible mistake: dictionary entry = LAST row of each tuple
    last = np.empty_like(first)
    for i, t in enumerate(ids.tolist()):
        last[t] = i
    return ids, last, d


def _ignore_unsigned(cols, unsigned_mask=0):
    return _real_map_tuples(cols, 0)


def _reverse_significance(cols, unsigned_mask=0):
    rev = list(cols)[::-1]
    m = 0
    for c in range(len(cols)):
        if (unsigned_mask >> c) & 1:
            m |= 1 << (len(cols) - 1 - c)
    return _real_map_tuples(rev, m)


def _keep_negative(r_y, r_x, s_y, s_z):
    return oracle.join_project(r_y, r_x, s_y, s_z)


def _keep_negative_count(r_y, r_x, s_y, s_z):
    return oracle.join_count(r_y, r_x, s_y, s_z)


_real_map_tuples = om.map_tuples

MAPPING_MUTATIONS = {
    "first_is_last_row": {"map_tuples": _unstable_order},
    "unsigned_ignored": {"map_tuples": _ignore_unsigned},
    "least_significant_first": {"map_tuples": _reverse_significance},
    "negatives_kept": {"join_project_ids": _keep_negative, "join_count_ids": _keep_negative_count},
}


@pytest.mark.parametrize("name", sorted(MAPPING_MUTATIONS))
def test_mutation_caught(name, monkeypatch):
    for fn, repl in MAPPING_MUTATIONS[name].items():
        monkeypatch.setattr(oracle, fn, repl)
    with pytest.raises(AssertionError):
        _all_pins()


def test_pins_pass_unmutated():
    _all_pins()


def test_all_small_tuples_exhaustive():
    """Every multiset of up to 4 rows over {-1, 0, 1}^2."""
    vals = [-1, 0, 1]
    cells = list(itertools.product(vals, vals))
    for n in range(0, 4):
        for rows in itertools.product(cells, repeat=n):
            a = np.array([r[0] for r in rows], np.int32)
            b = np.array([r[1] for r in rows], np.int32)
            ids, first, _ = oracle.map_tuples([a, b])
            bids, bfirst = brute_map(list(rows))
            assert ids.tolist() == bids and first.tolist() == bfirst
