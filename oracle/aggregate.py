"""Join-Aggregate (Section 4.1) from its definition (test infrastructure only).

* ``join_aggregate``: group-by attributes from both tables,
  G_{x,z} agg(f(R.v, S.u)) over R(x, y, v) join_y S(z, y, u).
* ``groupby_aggregate``: group-by attribute from one table,
  G_x agg(z) over R(x, y) join_y S(z, y).

Readings: R and S are bags of rows (SQL semantics: every pair of rows with
equal y is one join tuple, duplicate rows included); values are int32;
f(v, u) is one of v * u, v + u, v, u, evaluated in int64; agg is COUNT, SUM,
MIN, MAX (int64 results, SUM wrapping modulo 2^64) or AVG (float64 division
of the int64 SUM by the COUNT). Groups are the (x, z) (or x) with at least
one join tuple, in canonical (ascending) order.

Plain definition: the join tuples are materialised (every R row paired with
every S row of its y), f is applied to each, and the tuples are grouped and
reduced with numpy.
"""

from __future__ import annotations

import numpy as np

AGGS = ("count", "sum", "min", "max", "avg")
FNS = ("mul", "add", "left", "right")


def _join_rows(r_key, s_key):
    """(ri, si): index pairs of all R and S rows with equal y."""
    r_key = np.asarray(r_key, np.int64)
    s_key = np.asarray(s_key, np.int64)
    order = np.argsort(s_key, kind="stable")
    sk = s_key[order]
    lo = np.searchsorted(sk, r_key, "left")
    hi = np.searchsorted(sk, r_key, "right")
    cnt = hi - lo
    ri = np.repeat(np.arange(r_key.size), cnt)
    starts = np.repeat(lo, cnt)
    within = np.arange(ri.size) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    si = order[starts + within]
    return ri, si


def _reduce(keys, vals, agg):
    """Group by the key columns (lexicographic), reduce vals: (group keys, result)."""
    if vals.size == 0:
        return [k[:0] for k in keys], (np.zeros(0, np.float64) if agg == "avg" else np.zeros(0, np.int64))
    order = np.lexsort(tuple(keys[::-1]))
    ks = [k[order] for k in keys]
    v = vals[order]
    diff = np.zeros(v.size, bool)
    diff[0] = True
    for k in ks:
        diff[1:] |= k[1:] != k[:-1]
    starts = np.flatnonzero(diff)
    counts = np.diff(np.append(starts, v.size))
    with np.errstate(over="ignore"):
        if agg == "count":
            res = counts.astype(np.int64)
        elif agg == "sum":
            res = np.add.reduceat(v, starts)
        elif agg == "min":
            res = np.minimum.reduceat(v, starts)
        elif agg == "max":
            res = np.maximum.reduceat(v, starts)
        elif agg == "avg":
            res = np.add.reduceat(v, starts).astype(np.float64) / counts.astype(np.float64)
        else:
            raise ValueError(agg)
    return [k[starts] for k in ks], res


def _f(v, u, fn):
    v = v.astype(np.int64)
    u = u.astype(np.int64)
    with np.errstate(over="ignore"):
        if fn == "mul":
            return v * u
        if fn == "add":
            return v + u
        if fn == "left":
            return v
        if fn == "right":
            return u
    raise ValueError(fn)


def join_aggregate(r_key, r_val, r_v, s_key, s_val, s_u, agg: str, fn: str):
    """(x, z, result) of G_{x,z} agg(f(R.v, S.u)) (R(x=r_val, y=r_key, v), S(z=s_val, y=s_key, u))."""
    r_val, r_v = np.asarray(r_val, np.int32), np.asarray(r_v, np.int32)
    s_val, s_u = np.asarray(s_val, np.int32), np.asarray(s_u, np.int32)
    ri, si = _join_rows(r_key, s_key)
    vals = _f(r_v[ri], s_u[si], fn)
    (x, z), res = _reduce([r_val[ri], s_val[si]], vals, agg)
    return x.astype(np.int32), z.astype(np.int32), res


def groupby_aggregate(r_key, r_val, s_key, s_val, agg: str):
    """(x, result) of G_x agg(z) over R(x=r_val, y=r_key) join_y S(z=s_val, y=s_key)."""
    r_val = np.asarray(r_val, np.int32)
    s_val = np.asarray(s_val, np.int32)
    ri, si = _join_rows(r_key, s_key)
    (x,), res = _reduce([r_val[ri]], s_val[si].astype(np.int64), agg)
    return x.astype(np.int32), res
