"""Seeded synthetic inputs drawn on a CUDA device with torch.

The same recipes as ``synth.py`` (pools of random distinct 32-bit ids, Zipf
join keys by inverse-CDF sampling, distinct tuples topped up to the stated
count, a random subset in random order), drawn with a seeded torch generator
on the device. It serves workloads too large to draw on the host in seconds:
the 2,000-query stream (about 7.7e8 tuples per table in all) takes minutes in
numpy and seconds here. The draws differ from ``synth.py``'s (another random
generator), the distributions do not. A given seed gives the same tables for a
given torch build and GPU.

Nothing here computes a join, a mapping, a partition or an output: it only
draws numbers and removes duplicate input tuples.
"""

from __future__ import annotations

import torch

_U32 = 1 << 32


def generator(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _as_i32(v: torch.Tensor) -> torch.Tensor:
    """int64 values in [0, 2^32) as the int32 with the same 32 bits."""
    return torch.where(v >= (1 << 31), v - _U32, v).to(torch.int32)


def random_ids(g: torch.Generator, k: int, device) -> torch.Tensor:
    """k distinct uniformly random 32-bit values, in random order, as int32."""
    out = torch.empty(0, dtype=torch.int64, device=device)
    while out.numel() < k:
        n = int((k - out.numel()) * 1.05) + 16
        draw = torch.randint(0, _U32, (n,), generator=g, device=device, dtype=torch.int64)
        out = torch.unique(torch.cat([out, draw]))
    perm = torch.randperm(out.numel(), generator=g, device=device)[:k]
    return _as_i32(out[perm])


def zipf_ranks(g: torch.Generator, n_ranks: int, s: float, size: int, device) -> torch.Tensor:
    """size draws from a bounded Zipf law over ranks 0..n_ranks-1, P(rank r)
    proportional to 1/(r+1)^s, by inverse-CDF sampling (int64)."""
    w = 1.0 / torch.arange(1, n_ranks + 1, dtype=torch.float64, device=device) ** s
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    u = torch.rand(size, generator=g, dtype=torch.float64, device=device)
    return torch.searchsorted(cdf, u, right=True).clamp_(max=n_ranks - 1)


def distinct_pairs(g: torch.Generator, n: int, draw, device, max_rounds: int = 200):
    """Call ``draw(k) -> (a, b)`` (int32 tensors) until n distinct (a, b)
    pairs exist; return n of them (a random subset) in random order."""
    keys = torch.empty(0, dtype=torch.int64, device=device)
    for _ in range(max_rounds):
        if keys.numel() >= n:
            break
        a, b = draw(int((n - keys.numel()) * 1.25) + 64)
        k = (a.to(torch.int64) << 32) | (b.to(torch.int64) & (_U32 - 1))
        keys = torch.unique(torch.cat([keys, k]))
    else:
        raise RuntimeError(f"could not draw {n} distinct tuples")
    keys = keys[torch.randperm(keys.numel(), generator=g, device=device)[:n]]
    return (keys >> 32).to(torch.int32), _as_i32(keys & (_U32 - 1))


def two_table(seed: int, n_r: int, n_s: int, nx: int, nz: int, ny: int, s_zipf: float, device):
    """R(x, y), S(z, y) on the device: x uniform over nx random ids, z uniform
    over nz, y Zipf(s_zipf) over ny ids shared by both tables. Returns the
    columns (r_key, r_val, s_key, s_val) as int32 device tensors."""
    g = generator(seed, device)
    xpool, zpool, ypool = random_ids(g, nx, device), random_ids(g, nz, device), random_ids(g, ny, device)

    def draw_r(k):
        return xpool[torch.randint(0, nx, (k,), generator=g, device=device)], ypool[zipf_ranks(g, ny, s_zipf, k, device)]

    def draw_s(k):
        return zpool[torch.randint(0, nz, (k,), generator=g, device=device)], ypool[zipf_ranks(g, ny, s_zipf, k, device)]

    rx, ry = distinct_pairs(g, n_r, draw_r, device)
    sz, sy = distinct_pairs(g, n_s, draw_s, device)
    return ry, rx, sy, sz


def query_tables(q, device):
    """The tables of one query of ``synth.config5_stream`` (t tuples per
    table, |X| = t/10, |Z| = t/12.5, |Y| = t/20, Zipf 1.0), drawn on the
    device from the query's seed."""
    t = q.tuples
    return two_table(q.seed, t, t, max(2, t // 10), max(2, int(t / 12.5)), max(2, t // 20), 1.0, device)
