"""Pins of the MJP oracle (Section 4.2, ``oracle/mjp.py``).

From outside the oracle's code: path enumeration over tiny graphs (the line
query's result and its bag and set sizes), a forward simulation of every
deduplication placement of a left-deep plan under the same cost model and
size assumption (the DP must find the cheapest, and its placement must cost
what the DP says), and a small example worked by hand. Planted mistakes in a
copy of the DP must be caught.
"""

import itertools

import numpy as np
import pytest

import oracle
import oracle.mjp as om


def rand_tables(seed, k, n=12, span=5):
    rng = np.random.default_rng(seed)
    return [(rng.integers(-span, span, n), rng.integers(-span, span, n)) for _ in range(k)]


def brute_paths(tables):
    """All join paths (as tuples of values) of the line query over set relations."""
    rels = [sorted(set(zip(map(int, a), map(int, b)))) for a, b in tables]
    paths = [[u, v] for u, v in rels[0]]
    sizes_j, sizes_p = [len(paths)], [len({(p[0], p[-1]) for p in paths})]
    for rel in rels[1:]:
        paths = [p + [v] for p in paths for (u, v) in rel if u == p[-1]]
        sizes_j.append(len(paths))
        sizes_p.append(len({(p[0], p[-1]) for p in paths}))
    return paths, sizes_j, sizes_p


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_line_query_bruteforce(seed, k):
    tables = rand_tables(seed, k)
    paths, sj, sp = brute_paths(tables)
    x, z = oracle.line_join_project(tables)
    assert list(zip(x.tolist(), z.tolist())) == sorted({(p[0], p[-1]) for p in paths})
    out_j, out_p = oracle.chain_sizes(tables)
    assert out_j == [float(v) for v in sj] and out_p == [float(v) for v in sp]


def simulate(r_size, out_j, out_p, c, dedup):
    """Cost of a left-deep plan with deduplications after the joins flagged in
    dedup (0-based table index; the last must be set), walking forward."""
    cost, last = 0.0, 0
    for h in range(1, len(r_size)):
        rho = out_p[last] / out_j[last] if out_j[last] > 0 else 0.0
        left, right = rho * out_j[h - 1], r_size[h]
        if dedup[h]:
            cost += c[2] * (left + right) + c[3] * rho * out_j[h] + c[4] * out_p[h]
            last = h
        else:
            cost += c[0] * (left + right) + c[1] * rho * out_j[h]
    return cost


@pytest.mark.parametrize("seed", range(40))
def test_dp_is_optimal(seed):
    rng = np.random.default_rng(900 + seed)
    k = int(rng.integers(2, 8))
    r_size = rng.integers(1, 10**6, k).astype(float).tolist()
    out_j = [r_size[0]]
    out_p = [r_size[0]]
    for _ in range(1, k):
        out_j.append(float(out_j[-1] * rng.uniform(0.5, 40)))
        out_p.append(float(min(out_j[-1], out_j[-1] * rng.uniform(0.01, 1.0))))
    c = rng.uniform(0.1, 5, 5).tolist()
    best, dedup = oracle.mjp_dp(r_size, out_j, out_p, c)
    assert dedup[-1]
    brute = min(simulate(r_size, out_j, out_p, c, [False] + list(m) + [True])
                for m in itertools.product([False, True], repeat=k - 2))
    assert best == pytest.approx(brute, rel=1e-12)
    assert simulate(r_size, out_j, out_p, c, dedup) == pytest.approx(best, rel=1e-12)


def test_worked_example():
    """Three tables worked by hand (all constants 1): rho = (1, 2/3, 2/3);
    DP_2 = (3 + 2) + 3 + 2 = 10; DP_3 = min(j = 1: join 8 + JP 9 = 17,
    j = 2: 10 + JP 7 = 17) = 17, the tie going to the plan without the middle
    deduplication."""
    t = [(np.array([1, 1, 2]), np.array([10, 11, 10])), (np.array([10, 11]), np.array([20, 20])),
         (np.array([20]), np.array([30]))]
    out_j, out_p = oracle.chain_sizes(t)
    assert out_j == [3.0, 3.0, 3.0] and out_p == [3.0, 2.0, 2.0]
    best, dedup = oracle.mjp_dp([3.0, 2.0, 1.0], out_j, out_p, [1, 1, 1, 1, 1])
    assert best == 17.0 and dedup == [False, False, True]
    # costlier output writes make the middle deduplication pay
    best, dedup = oracle.mjp_dp([3.0, 2.0, 1.0], [3.0, 30.0, 300.0], [3.0, 2.0, 2.0], [1, 1, 1, 1, 1])
    assert dedup == [False, True, True]


# ---------------------------------------------------------------- mutations
_real_dp = om.dp


def _no_rho(r_size, out_j, out_p, c):
    return _real_dp(r_size, out_j, [v for v in out_j], c)


def _skip_middle_joins(r_size, out_j, out_p, c):
    k = len(r_size)
    best, dedup = _real_dp(r_size, out_j, out_p, [c[0], c[1], c[2], c[3], c[4]])
    # plausible mistake: always deduplicate after every join
    return best, [False] + [True] * (k - 1)


MUTATIONS = {"rho_ignored": _no_rho, "dedup_everywhere": _skip_middle_joins}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_caught(name, monkeypatch):
    monkeypatch.setattr(oracle, "mjp_dp", MUTATIONS[name])
    with pytest.raises(AssertionError):
        for s in range(40):
            test_dp_is_optimal(s)
        test_worked_example()
