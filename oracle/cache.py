"""Partial result caching (Section 3), from its definitions (test
infrastructure only).

Definitions and the readings taken where the section leaves room:

* For a set Z_cached of z values, the cached partial results are
  R_cached = {(x, z) in the result of Eq. 1 : z in Z_cached}.
* Per z, k(z) = |{x : (x, z) in the result}|. The entry of a cached z is
  (z, size, x_1 .. x_j): the x list itself when k <= |X| / 2 (size = k), the
  complement X minus that list when k > |X| / 2 (size = k - |X| < 0). The
  size's sign cannot mark a complement when k = |X| (size 0, as for an empty
  list), so every entry also carries an explicit complement flag.
  space(z) = 2 + min(k, |X| - k). |X| is the plan's x dictionary: the x of R
  tuples whose y occurs in S.y.
* cost(z) restates the section's statistic (times z is touched by the inner
  loops, times per-touch constants) for this GPU path: a sparse z is touched
  once per join tuple through it, n_join(z) = sum over the S tuples (z, y) of
  deg_R(y), so cost = n_join(z) * t_sparse; a dense z (m_z >= theta_z) is
  evaluated once per x by DenseEC, so cost = |X| * t_dense.
* CacheScore(z) = cost(z) / space(z), in float64. The z are ranked by
  descending score, ties by ascending z value, and Z_cached is the longest
  prefix of that ranking whose total space is at most the budget B.
* A run with the cache removes the S tuples of cached z after mapping (so
  the dictionaries do not change), computes the rest as usual and adds
  R_cached; the union is the full result.

Plain numpy over the classical oracle; no blocking or reordering beyond the
definitions above.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from .core import join_project
from .plan import plan


@dataclasses.dataclass
class CacheStats:
    dict_x: np.ndarray   # |X| x values ascending
    dict_z: np.ndarray   # z values ascending
    k: np.ndarray        # per z: result x count
    n_join: np.ndarray   # per z: join tuples through z
    dense: np.ndarray    # per z: m_z >= theta_z


@dataclasses.dataclass
class Cache:
    n_x: int
    z: np.ndarray        # cached z values, ascending
    size: np.ndarray     # int64 per entry: k, or k - |X| for a complement entry
    complement: np.ndarray  # bool per entry
    offsets: np.ndarray  # int64 [n_entries + 1] into xs
    xs: np.ndarray       # int32: each entry's x list or complement, ascending


def cache_stats(r_key, r_val, s_key, s_val, theta_z: int) -> CacheStats:
    p = plan(r_key, r_val, s_key, s_val, theta_z)
    _, z, _ = join_project(r_key, r_val, s_key, s_val)
    k = np.bincount(np.searchsorted(p.dict_z, z), minlength=p.dict_z.size).astype(np.int64)
    # n_join(z): over the distinct S tuples (z, y), deg_R(y) summed per z
    s_y = np.asarray(s_key, np.int32)
    s_z = np.asarray(s_val, np.int32)
    packed = np.unique((s_z.astype(np.int64) << 32) | (s_y.astype(np.int64) & 0xFFFFFFFF))
    sz = (packed >> 32).astype(np.int32)
    sy = (packed & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
    z_id = np.searchsorted(p.dict_z, sz)
    y_id = np.searchsorted(p.dict_y, sy)
    n_join = np.bincount(z_id, weights=p.deg_r[y_id].astype(np.float64), minlength=p.dict_z.size)
    return CacheStats(dict_x=p.dict_x, dict_z=p.dict_z, k=k, n_join=n_join.astype(np.int64),
                      dense=p.dense_z.copy())


def cache_scores(st: CacheStats, t_sparse: float, t_dense: float):
    """(cost, space, score) per z, float64 / int64 / float64."""
    n_x = st.dict_x.size
    space = 2 + np.minimum(st.k, n_x - st.k)
    cost = np.where(st.dense, float(n_x) * t_dense, st.n_join.astype(np.float64) * t_sparse)
    return cost, space, cost / space


def cache_select(st: CacheStats, budget: int, t_sparse: float, t_dense: float) -> np.ndarray:
    """Indices (into dict_z) of Z_cached, ascending."""
    _, space, score = cache_scores(st, t_sparse, t_dense)
    rank = np.lexsort((st.dict_z, -score))  # primary: score descending; ties: z ascending
    total = np.cumsum(space[rank])
    n_take = int(np.searchsorted(total, budget, side="right"))
    return np.sort(rank[:n_take])


def cache_build(r_key, r_val, s_key, s_val, theta_z: int, budget: int, t_sparse: float,
                t_dense: float) -> Cache:
    st = cache_stats(r_key, r_val, s_key, s_val, theta_z)
    sel = cache_select(st, budget, t_sparse, t_dense)
    x, z, _ = join_project(r_key, r_val, s_key, s_val)
    by_z = np.lexsort((x, z))  # the result grouped by z, x ascending within a z
    xg, zg = x[by_z], z[by_z]
    n_x = st.dict_x.size
    sizes, lists, comp = [], [], []
    for i in sel:
        lo, hi = np.searchsorted(zg, st.dict_z[i], "left"), np.searchsorted(zg, st.dict_z[i], "right")
        xs = xg[lo:hi]
        if xs.size > n_x / 2:
            lists.append(np.setdiff1d(st.dict_x, xs))
            sizes.append(xs.size - n_x)
            comp.append(True)
        else:
            lists.append(xs)
            sizes.append(xs.size)
            comp.append(False)
    offsets = np.zeros(len(lists) + 1, np.int64)
    offsets[1:] = np.cumsum([a.size for a in lists])
    xs = np.concatenate(lists).astype(np.int32) if lists else np.zeros(0, np.int32)
    return Cache(n_x=n_x, z=st.dict_z[sel].astype(np.int32), size=np.asarray(sizes, np.int64),
                 complement=np.asarray(comp, bool), offsets=offsets, xs=xs)


def cached_pairs(c: Cache, dict_x: np.ndarray):
    """R_cached expanded to (x, z) pairs (canonical order)."""
    xs, zs = [], []
    for e in range(c.z.size):
        lst = c.xs[c.offsets[e]:c.offsets[e + 1]]
        full = np.setdiff1d(dict_x, lst) if c.complement[e] else lst
        xs.append(full)
        zs.append(np.full(full.size, c.z[e], np.int32))
    if not xs:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    x, z = np.concatenate(xs).astype(np.int32), np.concatenate(zs)
    order = np.lexsort((z, x))
    return x[order], z[order]


def join_project_cached(r_key, r_val, s_key, s_val, c: Cache):
    """DIM^3 with cached partial results: Eq. 1 over R and the S tuples whose
    z is not cached, plus R_cached."""
    s_key = np.asarray(s_key, np.int32)
    s_val = np.asarray(s_val, np.int32)
    keep = ~np.isin(s_val, c.z)
    x1, z1, _ = join_project(r_key, r_val, s_key[keep], s_val[keep])
    p = plan(r_key, r_val, s_key, s_val, 1 << 30)  # dictionaries of the full tables
    x2, z2 = cached_pairs(c, p.dict_x)
    x, z = np.concatenate([x1, x2]), np.concatenate([z1, z2])
    order = np.lexsort((z, x))
    return x[order].astype(np.int32), z[order].astype(np.int32)
