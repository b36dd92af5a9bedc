"""Autotuner for the dense/sparse split and the DenseEC variant.

The paper chooses per z between SparseBMM and DenseEC with f2, and per
(x, z) between the SIMD and the probe method with f3, from cost constants
"measured in advance" (Section 2.6). On the GPU the same choices are made by
measurement on the input itself:

* candidates for theta_z (z is dense iff m_z >= theta_z) are infinity (all
  sparse) and the degrees at which the densest 0.1%, 1%, 5%, 20% and 100% of
  the z columns become dense;
* a (threshold, DenseEC variant) is skipped without running when it is
  clearly hopeless: a lower bound of its DenseEC time (the tensor-core
  product 2 |X| K |Z_d| at the measured fp8 rate, AND + popc word pairs, or
  the probe's words; K bounded by the dense tuples) is above twice the best
  time so far, or its operands would not fit a memory budget;
* every surviving (theta_z, DenseEC variant -- for the tensor-core variant
  also the tile width, 128 x 256 or 128 x 128 --, emit rows per CTA) is timed
  on the device (CUDA events around the one-call path) and the fastest wins.

Results are cached per GPU and input shape bucket (log2 of |R|, |S|, |X|,
|Y|, |Z| and of the largest m_z) in a JSON file, so a workload of the same
shape reuses the decision without re-timing. Every choice gives the same
result (the split is intersection-free, the variants are exact).
"""

from __future__ import annotations

import json
import math
import os
import threading

import numpy as np
import torch

from . import dim3

INF = (1 << 31) - 1
TC_FLOPS = 2.9e15           # sustained tensor rate of the DenseEC kernel (measured, fp8 0/1)
DENSE_BYTES_BUDGET = 16 << 30
_lock = threading.Lock()


def default_cache_path() -> str:
    base = os.environ.get("DIM3_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "dim3")
    return os.path.join(base, "tune.json") if not base.endswith(".json") else base


def shape_key(info: dict, m_z_max: int) -> str:
    lg = lambda v: int(math.log2(max(int(v), 1)))  # noqa: E731
    dev = torch.cuda.get_device_name()
    return f"{dev}|r{lg(info['n_r'])}|s{lg(info['n_s'])}|x{lg(info['n_x'])}|y{lg(info['n_y'])}|z{lg(info['n_z'])}" \
           f"|m{lg(m_z_max)}"


def theta_candidates(m_z: np.ndarray) -> list:
    if m_z.size == 0:
        return [INF]
    desc = np.sort(m_z)[::-1]
    out = [INF]
    for f in (0.001, 0.01, 0.05, 0.2, 1.0):
        k = max(1, int(math.ceil(f * desc.size)))
        out.append(int(desc[k - 1]))
    return sorted(set(out), reverse=True)


def dense_estimate(m_z: np.ndarray, theta: int, n_x: int, n_y: int):
    """Upper bounds of the DenseEC work and operand bytes for a threshold."""
    dense = m_z >= theta
    n_zd = int(dense.sum())
    k = min(int(n_y), int(m_z[dense].sum()))
    flops = 2.0 * n_x * k * n_zd
    k_pad = -(-k // 128) * 128
    bytes_ = (n_x + 256) * k_pad + (n_zd + 256) * k_pad
    return n_zd, flops, bytes_


POPC_WORDS = 1.3e13   # 32-bit AND + popc word operations per second (CUDA cores)
PROBE_WORDS = 1.0e13  # dense-index words OR-ed per second by the probe (L2 loads)


def variant_estimates(m_z: np.ndarray, theta: int, n_x: int, n_y: int, n_r: int) -> dict:
    """Per DenseEC variant, (lower-bound seconds, operand bytes) for a
    threshold: the tensor-core product (2 |X| K |Z_d| FLOP, 0/1 bytes of R
    and S over K), AND + popc (|X| |Z_d| ceil(K / 32) word pairs, bitmaps of
    R and S over K) and the probe (each R entry ORs one row of ceil(|Z_d| /
    32) words, S's rows over the dense index). Every variant also holds the
    dense result bits, |X| ceil(|Z_d| / 32) words."""
    n_zd, flops, tc_bytes = dense_estimate(m_z, theta, n_x, n_y)
    if n_zd == 0:
        return {}
    k = min(int(n_y), int(m_z[m_z >= theta].sum()))
    kw, zdw = -(-k // 32), -(-n_zd // 32)
    res = n_x * zdw * 4
    return {dim3.DENSE_TC: (flops / TC_FLOPS, tc_bytes + res),
            dim3.DENSE_POPC: (n_x * n_zd * kw / POPC_WORDS, (n_x + n_zd) * kw * 4 + res),
            dim3.DENSE_PROBE: (n_r * zdw / PROBE_WORDS, k * zdw * 4 + res)}


def _time_join(ctx, cols, out_x, out_z, repeats: int, batch: bool = False) -> float:
    def call():
        if batch:
            ctx.batch_join_project(cols, out_x=out_x, out_z=out_z)
        else:
            ctx.join_project(*cols, out_x=out_x, out_z=out_z)

    call()  # warm
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        call()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(ctx: dim3.Context, cols, repeats: int = 2, cache_path: str | None = None, use_cache: bool = True,
         apply: bool = True, batch: bool = False) -> dict:
    """Choose theta_z, the DenseEC variant and the emit rows per CTA for the
    input `cols` = (r_key, r_val, s_key, s_val) on device -- or, with batch,
    a list of such instances timed through one batched call; set them on
    `ctx` (apply) and return the decision with the timings it rests on."""
    plan = ctx.batch_partition(cols, theta_z=INF) if batch else ctx.partition(*cols, theta_z=INF)
    info = plan.info
    m_z = plan.export("m_z").cpu().numpy().astype(np.int64)
    out_p = int(plan.row_counts().sum().item())
    plan.close()
    key = shape_key(info, int(m_z.max()) if m_z.size else 0) + ("|batch" if batch else "")
    path = cache_path or default_cache_path()
    if use_cache:
        with _lock:
            try:
                cached = json.load(open(path)).get(key)
            except Exception:  # noqa: BLE001
                cached = None
        if cached:
            if apply:
                _apply(ctx, cached)
            return dict(cached, cached=True)

    out_x = torch.empty(max(out_p, 1), dtype=torch.int32, device=ctx.device)
    out_z = torch.empty(max(out_p, 1), dtype=torch.int32, device=ctx.device)
    trials = []
    best = None
    for theta in theta_candidates(m_z):
        est = variant_estimates(m_z, theta, info["n_x"], info["n_y"], info["n_r_kept"])
        n_zd = int((m_z >= theta).sum())
        variants = [dim3.DENSE_AUTO] if n_zd == 0 else []
        for v, (sec, nbytes) in est.items():
            if nbytes > DENSE_BYTES_BUDGET:
                trials.append({"theta": theta, "variant": int(v), "skipped": "dense operands over budget",
                               "n_zd": n_zd, "bytes": nbytes})
            elif best is not None and sec * 1e3 > 2 * best["ms"]:
                trials.append({"theta": theta, "variant": int(v), "skipped": "DenseEC work above twice the best time",
                               "n_zd": n_zd, "est_ms": sec * 1e3})
            else:
                variants.append(v)
        shapes = [(v, tn) for v in variants for tn in ((256, 128) if v == dim3.DENSE_TC else (0,))]
        for v, tile_n in shapes:
            for rows in ((4, 2, 1) if batch else (2, 1)):
                cfg = {"theta": int(theta), "variant": int(v), "emit_rows": rows, "tile_n": tile_n}
                _apply(ctx, cfg)
                try:
                    ms = _time_join(ctx, cols, out_x, out_z, repeats, batch)
                except dim3.Dim3Error as e:
                    trials.append(dict(cfg, error=str(e)))
                    continue
                trials.append(dict(cfg, ms=ms, n_zd=n_zd))
                if best is None or ms < best["ms"]:
                    best = dict(cfg, ms=ms, n_zd=n_zd)
    del out_x, out_z
    decision = dict(best or {"theta": INF, "variant": 0, "emit_rows": 0, "ms": float("nan"), "n_zd": 0})
    decision["key"] = key
    decision["trials"] = trials
    if apply:
        _apply(ctx, decision)
    if use_cache:
        with _lock:
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                try:
                    data = json.load(open(path))
                except Exception:  # noqa: BLE001
                    data = {}
                data[key] = {k: decision.get(k, 0) for k in ("theta", "variant", "emit_rows", "tile_n", "ms", "n_zd")}
                tmp = path + f".tmp{os.getpid()}"
                json.dump(data, open(tmp, "w"), indent=1)
                os.replace(tmp, path)
            except OSError:
                pass
    return dict(decision, cached=False)


def _apply(ctx, cfg: dict):
    ctx.set_option(dim3.OPT_THETA_Z, int(cfg["theta"]))
    ctx.set_option(dim3.OPT_DENSE_VARIANT, int(cfg["variant"]))
    ctx.set_option(dim3.OPT_EMIT_ROWS, int(cfg.get("emit_rows", 0)))
    ctx.set_option(dim3.OPT_DENSE_TILE_N, int(cfg.get("tile_n", 0)))


VARIANT_NAMES = {dim3.DENSE_AUTO: "sparse", dim3.DENSE_TC: "tc", dim3.DENSE_POPC: "popc", dim3.DENSE_PROBE: "probe"}


def summary(decision: dict) -> dict:
    """The decision without its trial list, plus the number of candidates
    timed and skipped and the best time of every DenseEC choice
    ("sparse" = no dense z; "tc256" / "tc128" = the tensor-core product with
    128 x 256 / 128 x 128 tiles; "popc"; "probe") with its threshold, for a
    bench line's config."""
    trials = decision.get("trials", [])
    out = {k: v for k, v in decision.items() if k != "trials"}
    out["timed"] = sum(1 for t in trials if "ms" in t)
    out["skipped"] = sum(1 for t in trials if "skipped" in t)
    best = {}
    for t in trials:
        if "ms" not in t:
            continue
        name = VARIANT_NAMES.get(t["variant"], str(t["variant"])) if t.get("n_zd", 0) else "sparse"
        if name == "tc":
            name += str(t.get("tile_n", 256))
        if name not in best or t["ms"] < best[name]["ms"]:
            best[name] = {"ms": t["ms"], "theta": t["theta"], "n_zd": t.get("n_zd", 0)}
    out["best_by_choice"] = best
    return out
