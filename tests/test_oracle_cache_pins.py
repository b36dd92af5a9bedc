"""Pins of the partial-result-caching oracle (Section 3, ``oracle/cache.py``).

The pins come from outside the oracle's code: a small example worked by hand
from the section's definitions (``tests/golden/sec3_cache_example.txt``), brute
force of k(z) and n_join(z) with Python sets, and the defining invariant of a
cached run: DIM^3 over R and the uncached S tuples, plus the cached partial
results, is the full result of Eq. 1 -- for random instances, budgets and
thresholds. ``test_mutation_caught`` plants plausible mistakes and checks that
a pin fails.
"""

import os

import numpy as np
import pytest

import oracle
import oracle.cache as oc
from tests.test_oracle_pins import brute_force

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sec3_cache_example.txt")


def load_example():
    R, S, stat, cases, selects, entries = [], [], {}, {}, [], []
    for line in open(GOLDEN):
        t = line.split("#")[0].split()
        if not t:
            continue
        if t[0] == "R":
            R.append((int(t[1]), int(t[2])))
        elif t[0] == "S":
            S.append((int(t[1]), int(t[2])))
        elif t[0] == "STAT":
            stat[int(t[1])] = tuple(int(v) for v in t[2:])
        elif t[0] == "CASE":
            cases[t[1]] = (int(t[2]), float(t[3]), float(t[4]))
        elif t[0] == "SELECT":
            selects.append((t[1], int(t[2]), [int(v) for v in t[3:]]))
        elif t[0] == "ENTRY":
            entries.append((t[1], int(t[2]), int(t[3]), bool(int(t[4])), int(t[5]), [int(v) for v in t[6:]]))
    return R, S, stat, cases, selects, entries


def cols(R, S):
    r = np.array(R, np.int32).reshape(-1, 2)
    s = np.array(S, np.int32).reshape(-1, 2)
    return r[:, 1], r[:, 0], s[:, 1], s[:, 0]  # r_key = y, r_val = x, s_key = y, s_val = z


def test_worked_example_stats():
    R, S, stat, _, _, _ = load_example()
    st = oracle.cache_stats(*cols(R, S), 2)
    _, space, _ = oracle.cache_scores(st, 1.0, 1.0)
    assert st.dict_x.tolist() == [1, 2, 3, 4]
    got = {int(z): (int(k), int(n), int(sp)) for z, k, n, sp in zip(st.dict_z, st.k, st.n_join, space)}
    assert got == {z: (v[0], v[1], v[3]) for z, v in stat.items()}
    m_z = {z: v[2] for z, v in stat.items()}
    assert [bool(d) for d in st.dense] == [m_z[int(z)] >= 2 for z in st.dict_z]


def test_worked_example_selection():
    R, S, _, cases, selects, _ = load_example()
    for name, budget, want in selects:
        theta, ts, td = cases[name]
        st = oracle.cache_stats(*cols(R, S), theta)
        sel = oracle.cache_select(st, budget, ts, td)
        assert st.dict_z[sel].tolist() == want, (name, budget)


def test_worked_example_entries():
    R, S, _, cases, _, entries = load_example()
    by = {}
    for name, budget, z, comp, size, lst in entries:
        by.setdefault((name, budget), []).append((z, comp, size, lst))
    for (name, budget), want in by.items():
        theta, ts, td = cases[name]
        c = oracle.cache_build(*cols(R, S), theta, budget, ts, td)
        got = [(int(c.z[e]), bool(c.complement[e]), int(c.size[e]), c.xs[c.offsets[e]:c.offsets[e + 1]].tolist())
               for e in range(c.z.size)]
        assert got == want


def brute_stats(r_key, r_val, s_key, s_val):
    R = set(zip(map(int, r_val), map(int, r_key)))
    S = set(zip(map(int, s_val), map(int, s_key)))
    ys = {y for _, y in S}
    Rk = {(x, y) for x, y in R if y in ys}
    deg = {}
    for _, y in Rk:
        deg[y] = deg.get(y, 0) + 1
    out = {}
    for z in sorted({z for z, _ in S}):
        yz = {y for zz, y in S if zz == z}
        xs = {x for x, y in Rk if y in yz}
        out[z] = (len(xs), sum(deg.get(y, 0) for y in yz))
    return sorted({x for x, _ in Rk}), out


@pytest.mark.parametrize("seed", range(10))
def test_stats_bruteforce(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 50))
    r_key, r_val = rng.integers(0, 9, n), rng.integers(0, 12, n)
    s_key, s_val = rng.integers(0, 11, n), rng.integers(-5, 6, n)
    X, want = brute_stats(r_key, r_val, s_key, s_val)
    st = oracle.cache_stats(r_key, r_val, s_key, s_val, 3)
    assert st.dict_x.tolist() == X
    assert {int(z): (int(k), int(m)) for z, k, m in zip(st.dict_z, st.k, st.n_join)} == want


@pytest.mark.parametrize("seed", range(12))
def test_cached_run_is_the_full_result(seed):
    rng = np.random.default_rng(800 + seed)
    inst_n = int(rng.integers(1, 400))
    r_key, r_val = rng.integers(0, 30, inst_n), rng.integers(0, 25, inst_n)
    s_key, s_val = rng.integers(0, 30, inst_n), rng.integers(0, 40, inst_n)
    full = brute_force(r_key, r_val, s_key, s_val)
    fx = [a for a, _, _ in full]
    fz = [b for _, b, _ in full]
    theta = int(rng.integers(1, 6))
    for budget in (0, 5, 40, 200, 10**9):
        c = oracle.cache_build(r_key, r_val, s_key, s_val, theta, budget, 1.0, float(rng.uniform(0.01, 2)))
        x, z = oracle.join_project_cached(r_key, r_val, s_key, s_val, c)
        assert x.tolist() == fx and z.tolist() == fz
        # entries: complements exactly when k > |X| / 2; space within budget
        st = oracle.cache_stats(r_key, r_val, s_key, s_val, theta)
        n_x = st.dict_x.size
        used = 0
        for e in range(c.z.size):
            k = sum(1 for b in fz if b == c.z[e])
            assert bool(c.complement[e]) == (k > n_x / 2)
            assert c.size[e] == (k - n_x if c.complement[e] else k)
            used += 2 + min(k, n_x - k)
        assert used <= budget


# ---------------------------------------------------------------- mutations
def _all_pins():
    test_worked_example_stats()
    test_worked_example_selection()
    test_worked_example_entries()
    for s in range(10):
        test_stats_bruteforce(s)
    for s in range(12):
        test_cached_run_is_the_full_result(s)


_real = {n: getattr(oc, n) for n in ("cache_scores", "cache_select", "cache_build", "cached_pairs", "plan")}


def _space_no_header(st, ts, td):
    cost, space, _ = _real["cache_scores"](st, ts, td)
    return cost, space - 2, cost / np.maximum(space - 2, 1)


def _ties_descending(st, budget, ts, td):
    _, space, score = oc.cache_scores(st, ts, td)
    rank = np.lexsort((-st.dict_z, -score))
    total = np.cumsum(space[rank])
    return np.sort(rank[:int(np.searchsorted(total, budget, side="right"))])


def _complement_at_half(r_key, r_val, s_key, s_val, theta, budget, ts, td):
    c = _real["cache_build"](r_key, r_val, s_key, s_val, theta, budget, ts, td)
    n_x = c.n_x
    x, z, _ = oracle.join_project(r_key, r_val, s_key, s_val)
    st = oracle.cache_stats(r_key, r_val, s_key, s_val, theta)
    for e in range(c.z.size):
        k = int((z == c.z[e]).sum())
        if k == n_x / 2:  # plausible mistake: >= instead of >
            c.complement[e] = True
            c.size[e] = k - n_x
            lst = np.setdiff1d(st.dict_x, x[z == c.z[e]])
            c.xs = np.concatenate([c.xs[:c.offsets[e]], lst, c.xs[c.offsets[e + 1]:]]).astype(np.int32)
            d = lst.size - (c.offsets[e + 1] - c.offsets[e])
            c.offsets[e + 1:] += d
    return c


def _no_complement_decode(c, dict_x):
    xs, zs = [], []
    for e in range(c.z.size):
        lst = c.xs[c.offsets[e]:c.offsets[e + 1]]
        xs.append(lst)
        zs.append(np.full(lst.size, c.z[e], np.int32))
    if not xs:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    x, z = np.concatenate(xs).astype(np.int32), np.concatenate(zs)
    o = np.lexsort((z, x))
    return x[o], z[o]


def _stale_dictionary(r_key, r_val, s_key, s_val, c):
    # plausible mistake: X taken after the cached z's S tuples were removed
    s_key = np.asarray(s_key, np.int32)
    s_val = np.asarray(s_val, np.int32)
    keep = ~np.isin(s_val, c.z)
    x1, z1, _ = oracle.join_project(r_key, r_val, s_key[keep], s_val[keep])
    p = _real["plan"](r_key, r_val, s_key[keep], s_val[keep], 1 << 30)
    x2, z2 = oc.cached_pairs(c, p.dict_x)
    x, z = np.concatenate([x1, x2]), np.concatenate([z1, z2])
    o = np.lexsort((z, x))
    return x[o].astype(np.int32), z[o].astype(np.int32)


MUTATIONS = {
    "space_without_header": {"cache_scores": _space_no_header},
    "ties_by_z_descending": {"cache_select": _ties_descending},
    "complement_at_exactly_half": {"cache_build": _complement_at_half},
    "complement_not_decoded": {"cached_pairs": _no_complement_decode},
    "dictionary_of_reduced_s": {"join_project_cached": _stale_dictionary},
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_caught(name, monkeypatch):
    for fn, repl in MUTATIONS[name].items():
        monkeypatch.setattr(oc, fn, repl)
        if hasattr(oracle, fn):
            monkeypatch.setattr(oracle, fn, repl)
    with pytest.raises(AssertionError):
        _all_pins()


def test_pins_pass_unmutated():
    _all_pins()
