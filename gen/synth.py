"""Seeded synthetic Join-Project inputs.

The paper's real datasets (Table 2) are not available, so these generators
stand in for them. Their shapes follow the paper's own synthetic families:
uniform x/z, Zipf-distributed join keys y (Section 6, sensitivity to Zipf on
y) and power-law graphs (Section 6, R-MAT / power-law inputs). The tables are
made of distinct tuples, as in the paper's worst-case analysis, and are
shuffled, as the paper shuffles its inputs before every experiment
(Section 6.1).

Conventions: a table R(x, y) is two int32 columns ``r_val`` (x) and
``r_key`` (y); S(z, y) is ``s_val`` (z) and ``s_key`` (y). Ids are random
distinct 32-bit values viewed as int32, so they are non-contiguous and may be
negative.

Nothing here computes a join, a mapping, a partition or an output: it only
draws numbers and removes duplicate input tuples.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    """One Join-Project input: R(x, y) and S(z, y) as int32 columns."""

    name: str
    r_key: np.ndarray  # R.y
    r_val: np.ndarray  # R.x
    s_key: np.ndarray  # S.y
    s_val: np.ndarray  # S.z
    self_join: bool = False
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nr(self) -> int:
        return int(self.r_key.size)

    @property
    def ns(self) -> int:
        return int(self.s_key.size)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """The distinct values of a, ascending (np.unique's result, by one sort)."""
    a = np.sort(a, kind="stable")
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def random_ids(rng: np.random.Generator, k: int) -> np.ndarray:
    """k distinct uniformly random 32-bit values, in random order, as int32."""
    out = np.empty(0, dtype=np.uint32)
    while out.size < k:
        draw = rng.integers(0, 2**32, size=int((k - out.size) * 1.05) + 16,
                            dtype=np.uint64).astype(np.uint32)
        out = _sorted_unique(np.concatenate([out, draw]))
    return rng.permutation(out)[:k].view(np.int32)


def zipf_ranks(rng: np.random.Generator, n_ranks: int, s: float,
               size: int) -> np.ndarray:
    """size draws from a bounded Zipf law over ranks 0..n_ranks-1,
    P(rank r) proportional to 1/(r+1)^s, by inverse-CDF sampling."""
    w = 1.0 / np.arange(1, n_ranks + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    r = np.searchsorted(cdf, rng.random(size), side="right")
    return np.minimum(r, n_ranks - 1).astype(np.int64)


def _pack(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (a.astype(np.int64).astype(np.uint32).astype(np.uint64) << np.uint64(32)) | \
        b.astype(np.int64).astype(np.uint32).astype(np.uint64)


def _unpack(keys: np.ndarray):
    a = (keys >> np.uint64(32)).astype(np.uint32).view(np.int32)
    b = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    return a, b


def distinct_pairs(rng: np.random.Generator, n: int, draw, max_rounds: int = 200):
    """Call ``draw(rng, k) -> (a, b)`` until n distinct (a, b) pairs exist;
    return n of them (a random subset) in random order."""
    keys = np.empty(0, dtype=np.uint64)
    for _ in range(max_rounds):
        if keys.size >= n:
            break
        need = n - keys.size
        a, b = draw(rng, int(need * 1.25) + 64)
        keys = _sorted_unique(np.concatenate([keys, _pack(a, b)]))
    else:
        raise RuntimeError(f"could not draw {n} distinct tuples")
    keys = rng.permutation(keys)[:n]
    return _unpack(keys)


def two_table(rng: np.random.Generator, n_r: int, n_s: int, nx: int, nz: int,
              ny: int, s_zipf: float, name: str = "two_table") -> Instance:
    """R(x, y), S(z, y): x uniform over nx ids, z uniform over nz ids, y drawn
    Zipf(s_zipf) over ny ids shared by both tables."""
    xpool = random_ids(rng, nx)
    zpool = random_ids(rng, nz)
    ypool = random_ids(rng, ny)  # Zipf rank r -> ypool[r]; the pool is random

    def draw_r(g, k):
        return xpool[g.integers(0, nx, size=k)], ypool[zipf_ranks(g, ny, s_zipf, k)]

    def draw_s(g, k):
        return zpool[g.integers(0, nz, size=k)], ypool[zipf_ranks(g, ny, s_zipf, k)]

    rx, ry = distinct_pairs(rng, n_r, draw_r)
    sz, sy = distinct_pairs(rng, n_s, draw_s)
    return Instance(name, r_key=ry, r_val=rx, s_key=sy, s_val=sz,
                    meta=dict(n_r=n_r, n_s=n_s, nx=nx, nz=nz, ny=ny, s_zipf=s_zipf))


def config1_self(seed: int = 0) -> Instance:
    """Plain self Join-Project R = S: 20,000 distinct (x, y) tuples, x uniform
    over 2,000 random ids, y uniform over 1,000 random ids."""
    rng = np.random.default_rng(seed)
    xpool = random_ids(rng, 2000)
    ypool = random_ids(rng, 1000)

    def draw(g, k):
        return xpool[g.integers(0, 2000, size=k)], ypool[g.integers(0, 1000, size=k)]

    x, y = distinct_pairs(rng, 20000, draw)
    return Instance("self_20k", r_key=y, r_val=x, s_key=y, s_val=x, self_join=True,
                    meta=dict(n=20000, nx=2000, ny=1000, seed=seed))


def config2_two_table(seed: int = 1, scale: float = 1.0) -> Instance:
    """Two-table Join-Project, |R| = |S| = 1,000,000 distinct tuples; x uniform
    over 100,000 ids, z uniform over 80,000 ids, y Zipf(1.0) over 50,000 ids.
    ``scale`` shrinks every size proportionally (for tests)."""
    rng = np.random.default_rng(seed)
    n = int(round(1_000_000 * scale))
    inst = two_table(rng, n, n, max(1, int(100_000 * scale)),
                     max(1, int(80_000 * scale)), max(1, int(50_000 * scale)), 1.0,
                     name="two_table_1m_zipf1" if scale == 1.0 else f"two_table_zipf1_x{scale:g}")
    inst.meta["seed"] = seed
    return inst


def chung_lu_self(rng: np.random.Generator, n_vertices: int, n_edges: int,
                  beta: float, name: str = "chung_lu", cap: bool = True) -> Instance:
    """Self Join-Project over an undirected Chung-Lu power-law graph.

    Expected-degree weights w_i proportional to i^(-1/(beta-1)), scaled to sum
    2 * n_edges and, with cap, capped at sqrt(2 * n_edges) (the usual Chung-Lu
    constraint; without it the hubs keep their power-law weight); both
    endpoints of an edge are drawn proportionally to w. Self-loops and
    multi-edges are dropped and the draw is topped up to exactly n_edges
    edges. R = S holds both directions of every edge.
    """
    i = np.arange(1, n_vertices + 1, dtype=np.float64)
    w = i ** (-1.0 / (beta - 1.0))
    w *= 2.0 * n_edges / w.sum()
    if cap:
        w = np.minimum(w, math.sqrt(2.0 * n_edges))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]

    def draw(g, k):
        u = np.minimum(np.searchsorted(cdf, g.random(k), side="right"), n_vertices - 1)
        v = np.minimum(np.searchsorted(cdf, g.random(k), side="right"), n_vertices - 1)
        keep = u != v
        u, v = u[keep], v[keep]
        return np.minimum(u, v).astype(np.int32), np.maximum(u, v).astype(np.int32)

    lo, hi = distinct_pairs(rng, n_edges, draw)
    vid = random_ids(rng, n_vertices)
    x = np.concatenate([vid[lo], vid[hi]])
    y = np.concatenate([vid[hi], vid[lo]])
    perm = rng.permutation(x.size)
    x, y = x[perm], y[perm]
    return Instance(name, r_key=y, r_val=x, s_key=y, s_val=x, self_join=True,
                    meta=dict(n_vertices=n_vertices, n_edges=n_edges, beta=beta))


def config3_chung_lu(seed: int = 2, scale: float = 1.0) -> Instance:
    """Two-hop Join-Project over a Chung-Lu graph with 1,000,000 vertices,
    4,000,000 undirected edges and degree exponent 2.1."""
    rng = np.random.default_rng(seed)
    nv = max(16, int(1_000_000 * scale))
    ne = max(16, int(4_000_000 * scale))
    inst = chung_lu_self(rng, nv, ne, 2.1,
                         name="chung_lu_1m_4m" if scale == 1.0 else f"chung_lu_x{scale:g}")
    inst.meta["seed"] = seed
    return inst


def chung_lu_uncapped(seed: int = 2, scale: float = 1.0) -> Instance:
    """The Chung-Lu graph of config3_chung_lu without the weight cap (degree
    exponent 2.1, hubs with degrees near 10^5 at full size): a two-hop
    Join-Project whose hub z are dense enough for DenseEC. ``scale`` shrinks
    the vertex and edge counts proportionally."""
    rng = np.random.default_rng(seed)
    nv = max(16, int(1_000_000 * scale))
    ne = max(16, int(4_000_000 * scale))
    inst = chung_lu_self(rng, nv, ne, 2.1, cap=False,
                         name="chung_lu_uncapped_1m_4m" if scale == 1.0 else f"chung_lu_uncapped_x{scale:g}")
    inst.meta["seed"] = seed
    return inst


def batch_sizes(rng: np.random.Generator, n_inst: int, lo: int, hi: int) -> np.ndarray:
    """Tuple counts log-uniform in [lo, hi]."""
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_inst)).astype(np.int64)


def config4_batch(seed: int = 3, n_inst: int = 256, lo: int = 1000,
                  hi: int = 200_000) -> list[Instance]:
    """256 independent two-table instances: t tuples per table, log-uniform
    in [1,000, 200,000]; |Y| = t/20, |X| = t/10, |Z| = t/12.5; y Zipf(s),
    s uniform in [0.8, 1.2] per instance."""
    rng = np.random.default_rng(seed)
    ts = batch_sizes(rng, n_inst, lo, hi)
    ss = rng.uniform(0.8, 1.2, size=n_inst)
    out = []
    for k, (t, s) in enumerate(zip(ts, ss)):
        t = int(t)
        inst = two_table(rng, t, t, max(2, t // 10), max(2, int(t / 12.5)),
                         max(2, t // 20), float(s), name=f"batch{k}")
        out.append(inst)
    return out


@dataclasses.dataclass
class Query:
    arrival_s: float
    kind: str  # "project" or "count"
    tuples: int
    seed: int

    def instance(self) -> Instance:
        rng = np.random.default_rng(self.seed)
        t = self.tuples
        return two_table(rng, t, t, max(2, t // 10), max(2, int(t / 12.5)),
                         max(2, t // 20), 1.0, name=f"q{self.seed}")


def config5_stream(seed: int = 4, n_queries: int = 2000, rate_qps: float = 200.0,
                   lo: int = 10_000, hi: int = 2_000_000) -> list[Query]:
    """Poisson stream of Join-Project / Join-Count queries (50/50 by a seeded
    coin), tuple counts log-uniform in [lo, hi], Zipf(1.0) join keys."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_qps, size=n_queries)
    arrivals = np.cumsum(gaps)
    ts = batch_sizes(rng, n_queries, lo, hi)
    kinds = np.where(rng.random(n_queries) < 0.5, "project", "count")
    seeds = rng.integers(0, 2**31 - 1, size=n_queries)
    return [Query(float(a), str(k), int(t), int(s))
            for a, k, t, s in zip(arrivals, kinds, ts, seeds)]


def small_two_table(seed: int, n_r: int, n_s: int, nx: int, nz: int, ny: int,
                    dup_frac: float = 0.0, zipf: float | None = None,
                    self_join: bool = False) -> Instance:
    """Small random tables for tests. Values come from pools of random ids
    (so they are sparse and may be negative). With dup_frac > 0, that fraction
    of rows is repeated to exercise set semantics."""
    rng = np.random.default_rng(seed)
    xpool = random_ids(rng, nx)
    ypool = random_ids(rng, ny)
    zpool = xpool if self_join else random_ids(rng, nz)

    def ys(k):
        if zipf is None:
            return ypool[rng.integers(0, ny, size=k)]
        return ypool[zipf_ranks(rng, ny, zipf, k)]

    rx = xpool[rng.integers(0, nx, size=n_r)]
    ry = ys(n_r)
    if self_join:
        sz, sy = rx, ry
    else:
        sz = zpool[rng.integers(0, nz, size=n_s)]
        sy = ys(n_s)
    if dup_frac > 0 and n_r > 0:
        k = int(n_r * dup_frac)
        idx = rng.integers(0, n_r, size=k)
        rx = np.concatenate([rx, rx[idx]])
        ry = np.concatenate([ry, ry[idx]])
        if self_join:
            sz, sy = rx, ry
        elif n_s > 0:
            idx = rng.integers(0, n_s, size=int(n_s * dup_frac))
            sz = np.concatenate([sz, sz[idx]])
            sy = np.concatenate([sy, sy[idx]])
    return Instance(f"small{seed}", r_key=ry.astype(np.int32), r_val=rx.astype(np.int32),
                    s_key=sy.astype(np.int32), s_val=sz.astype(np.int32),
                    self_join=self_join)


CONFIGS = {
    "self_20k": config1_self,
    "two_table_1m_zipf1": config2_two_table,
    "chung_lu_1m_4m": config3_chung_lu,
    "batch256": config4_batch,
    "serve2000": config5_stream,
}
