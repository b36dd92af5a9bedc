"""Pins of the Join-Aggregate oracle (Section 4.1, ``oracle/aggregate.py``).

Each pin comes from outside the oracle's code: nested Python loops over the
row pairs of tiny bags (duplicates included), the classical Join-Count oracle
in C (COUNT over duplicate-free tables), and identities between aggregates
(SUM of v + u = SUM of v + SUM of u, MIN <= AVG <= MAX, the one-table query
as a fold of the two-table COUNT). ``test_mutation_caught`` plants plausible
mistakes and checks that a pin fails.
"""

import numpy as np
import pytest

import oracle
import oracle.aggregate as oa

AGGS = ("count", "sum", "min", "max", "avg")
FNS = ("mul", "add", "left", "right")


def brute_two(R, S, agg, fn):
    groups = {}
    for (x, y, v) in R:
        for (z, y2, u) in S:
            if y == y2:
                val = {"mul": v * u, "add": v + u, "left": v, "right": u}[fn]
                groups.setdefault((x, z), []).append(val)
    out = []
    for key in sorted(groups):
        g = groups[key]
        res = {"count": len(g), "sum": sum(g), "min": min(g), "max": max(g), "avg": sum(g) / len(g)}[agg]
        out.append((key[0], key[1], res))
    return out


def brute_one(R, S, agg):
    groups = {}
    for (x, y) in R:
        for (z, y2) in S:
            if y == y2:
                groups.setdefault(x, []).append(z)
    return [(x, {"count": len(g), "sum": sum(g), "min": min(g), "max": max(g), "avg": sum(g) / len(g)}[agg])
            for x, g in sorted(groups.items())]


def tiny(seed, n=25, dup=True):
    rng = np.random.default_rng(seed)
    R = [(int(rng.integers(0, 5)), int(rng.integers(0, 4)), int(rng.integers(-6, 7))) for _ in range(n)]
    S = [(int(rng.integers(-3, 3)), int(rng.integers(0, 4)), int(rng.integers(-6, 7))) for _ in range(n)]
    if dup:
        R += R[:4]
        S += S[:3]
    return R, S


def cols2(R, S):
    r = np.array(R, np.int64).reshape(-1, 3)
    s = np.array(S, np.int64).reshape(-1, 3)
    return r[:, 1], r[:, 0], r[:, 2], s[:, 1], s[:, 0], s[:, 2]


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("agg", AGGS)
@pytest.mark.parametrize("fn", FNS)
def test_two_table_bruteforce(seed, agg, fn):
    R, S = tiny(seed)
    x, z, res = oracle.join_aggregate(*cols2(R, S), agg, fn)
    got = list(zip(x.tolist(), z.tolist(), res.tolist()))
    assert got == brute_two(R, S, agg, fn)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("agg", AGGS)
def test_one_table_bruteforce(seed, agg):
    R, S = tiny(100 + seed)
    R2 = [(x, y) for x, y, _ in R]
    S2 = [(z, y) for z, y, _ in S]
    r = np.array(R2).reshape(-1, 2)
    s = np.array(S2).reshape(-1, 2)
    x, res = oracle.groupby_aggregate(r[:, 1], r[:, 0], s[:, 1], s[:, 0], agg)
    assert list(zip(x.tolist(), res.tolist())) == brute_one(R2, S2, agg)


@pytest.mark.parametrize("seed", range(5))
def test_count_matches_join_count(seed):
    """Without duplicate rows, COUNT of join tuples per (x, z) is the number of
    shared y: the classical Join-Count oracle (C)."""
    rng = np.random.default_rng(200 + seed)
    rk, rv = rng.integers(0, 40, 500), rng.integers(0, 60, 500)
    sk, sv = rng.integers(0, 40, 500), rng.integers(0, 50, 500)
    r = np.unique(np.stack([rk, rv], 1), axis=0)
    s = np.unique(np.stack([sk, sv], 1), axis=0)
    x, z, c = oracle.join_aggregate(r[:, 0], r[:, 1], np.ones(len(r)), s[:, 0], s[:, 1], np.ones(len(s)), "count",
                                    "mul")
    cx, cz, cc, _ = oracle.join_count(r[:, 0], r[:, 1], s[:, 0], s[:, 1])
    assert np.array_equal(x, cx) and np.array_equal(z, cz) and np.array_equal(c, cc)
    _, _, sm = oracle.join_aggregate(r[:, 0], r[:, 1], np.ones(len(r)), s[:, 0], s[:, 1], np.ones(len(s)), "sum",
                                     "mul")
    assert np.array_equal(sm, cc)


@pytest.mark.parametrize("seed", range(5))
def test_identities(seed):
    rng = np.random.default_rng(300 + seed)
    n = 800
    c = (rng.integers(0, 30, n), rng.integers(0, 40, n), rng.integers(-1000, 1000, n),
         rng.integers(0, 30, n), rng.integers(0, 35, n), rng.integers(-1000, 1000, n))
    _, _, s_add = oracle.join_aggregate(*c, "sum", "add")
    _, _, s_l = oracle.join_aggregate(*c, "sum", "left")
    _, _, s_r = oracle.join_aggregate(*c, "sum", "right")
    assert np.array_equal(s_add, s_l + s_r)
    for fn in FNS:
        _, _, mn = oracle.join_aggregate(*c, "min", fn)
        _, _, mx = oracle.join_aggregate(*c, "max", fn)
        _, _, av = oracle.join_aggregate(*c, "avg", fn)
        assert np.all(mn <= av) and np.all(av <= mx)
    # the one-table query folds the two-table COUNT: SUM(z) = sum_z z * COUNT(x, z)
    x2, z2, cnt = oracle.join_aggregate(*c, "count", "mul")
    x1, s1 = oracle.groupby_aggregate(c[0], c[1], c[3], c[4], "sum")
    fold = {}
    for a, b, k in zip(x2.tolist(), z2.tolist(), cnt.tolist()):
        fold[a] = fold.get(a, 0) + b * k
    assert list(zip(x1.tolist(), s1.tolist())) == sorted(fold.items())


# ---------------------------------------------------------------- mutations
def _all_pins():
    for s in range(8):
        for agg in AGGS:
            for fn in FNS:
                test_two_table_bruteforce(s, agg, fn)
            test_one_table_bruteforce(s, agg)
    for s in range(5):
        test_count_matches_join_count(s)
        test_identities(s)


_real_join_rows = oa._join_rows
_real_f = oa._f


def _set_semantics(r_key, s_key):
    # plausible mistake: a pair (R row's y, S row) joined once however many
    # identical R rows there are
    ri, si = _real_join_rows(r_key, s_key)
    rk = np.asarray(r_key)
    seen, keep = set(), np.ones(ri.size, bool)
    for i in range(ri.size):
        t = (int(rk[ri[i]]), int(si[i]))
        keep[i] = t not in seen
        seen.add(t)
    return ri[keep], si[keep]


def _add_as_mul(v, u, fn):
    return _real_f(v, u, "mul" if fn == "add" else fn)


def _swap_sides(v, u, fn):
    return _real_f(u, v, fn)


MUTATIONS = {
    "duplicates_joined_once": {"_join_rows": _set_semantics},
    "add_computed_as_mul": {"_f": _add_as_mul},
    "operands_swapped": {"_f": _swap_sides},
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_caught(name, monkeypatch):
    for fn, repl in MUTATIONS[name].items():
        monkeypatch.setattr(oa, fn, repl)
    with pytest.raises(AssertionError):
        _all_pins()


def test_pins_pass_unmutated():
    _all_pins()
