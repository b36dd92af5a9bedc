"""Multi-way joins with projection, MJP (Section 4.2), from the definitions
(test infrastructure only).

The line query Pi_{x_1, x_{k+1}}(R_1(x_1, x_2) join R_2(x_2, x_3) join ...
join R_k(x_k, x_{k+1})) over a left-deep plan, with deduplication placed
after some of the joins (always after the last).

* ``line_join_project``: the query's result, by deduplicating after every
  join with the classical oracle (any placement gives the same set).
* ``chain_sizes``: |OUT_J_i| = |R_1 join ... join R_i| (bag) and |OUT_P_i| =
  |Pi(OUT_J_i)|, i = 1..k, exactly (OUT_J_1 = OUT_P_1 = |R_1|).
* ``dp``: the dynamic programme of Section 4.2, in the paper's notation:
  DP_1 = 0; DP_i = min over j < i of DP_j + sum_{h=j+1}^{i-1} JoinCost_h +
  JPCost_i, where, after a deduplication at j, input sizes shrink by
  rho_j = |OUT_P_j| / |OUT_J_j| (assumption 4). Cost model (a GPU restatement
  of the section's cost formulas, five constants c):
    JoinCost(l, r, out)   = c0 (l + r) + c1 out            (bag join)
    JPCost(l, r, oj, op)  = c2 (l + r) + c3 oj + c4 op     (Join-Project)
  with l = rho_j |OUT_J_{h-1}|, r = |R_h|, out = rho_j |OUT_J_h| for a join
  and l = rho_j |OUT_J_{i-1}|, r = |R_i|, oj = rho_j |OUT_J_i|, op =
  |OUT_P_i| for the Join-Project at i. Ties take the smallest j. Returns
  (DP_k, dedup) with dedup[i] = True when a deduplication follows join i.

Relations are sets: duplicate input tuples collapse.
"""

from __future__ import annotations

import numpy as np

from .core import join_project


def _edges(t):
    a, b = t
    return np.asarray(a, np.int32), np.asarray(b, np.int32)


def line_join_project(tables):
    """(x_1, x_{k+1}) pairs of the line query, canonical (signed) order."""
    a, b = _edges(tables[0])
    if len(tables) == 1:
        order = np.lexsort((b, a))
        a, b = a[order], b[order]
        keep = np.ones(a.size, bool)
        keep[1:] = (a[1:] != a[:-1]) | (b[1:] != b[:-1])
        return a[keep], b[keep]
    x, z = a, b
    for t in tables[1:]:
        ta, tb = _edges(t)
        x, z, _ = join_project(z, x, ta, tb)  # R(x = x_1, y = current end), S(z = next, y = x_i)
    return x, z


def _distinct_edges(t):
    a, b = _edges(t)
    e = np.unique((a.astype(np.int64) << 32) | (b.astype(np.int64) & 0xFFFFFFFF))
    return (e >> 32).astype(np.int32), (e & 0xFFFFFFFF).astype(np.uint32).view(np.int32)


def chain_sizes(tables):
    """(out_j, out_p) lists of length k (float64)."""
    ea, eb = _distinct_edges(tables[0])
    out_j = [float(ea.size)]
    out_p = [float(ea.size)]
    # |OUT_J_i| as path counts: paths[v] = the number of join paths through
    # R_1 .. R_i ending at value v (Python integers, exact); the next table
    # extends every path ending at u along each of its edges (u, w)
    paths = {}
    for v in eb.tolist():
        paths[v] = paths.get(v, 0) + 1
    x, z = ea, eb
    for t in tables[1:]:
        ua, ub = _distinct_edges(t)
        nxt = {}
        for u, w in zip(ua.tolist(), ub.tolist()):
            c = paths.get(u, 0)
            if c:
                nxt[w] = nxt.get(w, 0) + c
        paths = nxt
        out_j.append(float(sum(paths.values())))
        x, z, _ = join_project(z, x, *_edges(t))
        out_p.append(float(x.size))
    return out_j, out_p


def dp(r_size, out_j, out_p, c):
    """(best cost, dedup flags) for tables 1..k (lists indexed 0..k-1)."""
    k = len(r_size)
    if k < 2:
        return 0.0, [False] * k
    rho = [out_p[i] / out_j[i] if out_j[i] > 0 else 0.0 for i in range(k)]

    def join_cost(l, r, out):
        return c[0] * (l + r) + c[1] * out

    def jp_cost(l, r, oj, op):
        return c[2] * (l + r) + c[3] * oj + c[4] * op

    best = [0.0] * k
    arg = [-1] * k
    for i in range(1, k):  # table index i (0-based) = the paper's i + 1
        cand = None
        for j in range(0, i):
            total = best[j]
            for h in range(j + 1, i):
                total += join_cost(rho[j] * out_j[h - 1], r_size[h], rho[j] * out_j[h])
            total += jp_cost(rho[j] * out_j[i - 1], r_size[i], rho[j] * out_j[i], out_p[i])
            if cand is None or total < cand:
                cand, arg[i] = total, j
        best[i] = cand
    dedup = [False] * k
    i = k - 1
    while i > 0:
        dedup[i] = True
        i = arg[i]
    return best[k - 1], dedup
