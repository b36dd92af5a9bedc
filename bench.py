#!/usr/bin/env python
"""Benchmark of the GB300 DIM^3 Join-Project hot path.

One step = one call of the C ABI's dim3_join_project on the two-table
workload (|R| = |S| = 10^6 distinct int32 tuples, 100,000 x, 80,000 z, Zipf(1.0)
y over 50,000 ids): mapping, partition, SparseBMM + DenseEC, union and
compaction of ~5e9 deduplicated (x, z) pairs into HBM. Inputs are resident in
HBM when the timed region starts.

Prints one JSON line (rank 0). With --impl reference it times the CPU oracle
instead (bounded samples of the same workload on the host cores).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "dedup (x,z) pairs/s on 1 GB300 vs plain path; served p50/p99 latency"
UNIT = "pairs/s"
WORKLOADS = ("two_table_1m_zipf1", "self_20k", "chung_lu_1m_4m", "chung_lu_uncapped_x0.25", "dense_16k", "batch256",
             "serve2000")
# fp8 (f8f6f4) dense tensor rate = 2 x bf16 (nominal 4.5 vs 2.25 PFLOP/s)
FP8_PER_BF16 = 2.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="two_table_1m_zipf1")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload proportionally (profiling captures only; bench lines use 1.0)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--theta-z", type=int, default=None, help="dense iff m_z >= theta (default: library's)")
    ap.add_argument("--dense-variant", type=int, default=None, help="0 auto, 1 tensor core, 2 popc, 3 probe")
    ap.add_argument("--opt", action="append", default=[],
                    help="library option KEY=VALUE (dim3_option number), e.g. 6=1 for one x row per emitting CTA")
    ap.add_argument("--batch-insts", type=int, default=256,
                    help="batch256: instances drawn (fewer for small profiling runs; the first ones of the stream)")
    ap.add_argument("--serve-queries", type=int, default=2000)
    ap.add_argument("--serve-max-tuples", type=int, default=2_000_000)
    ap.add_argument("--serve-workers", type=int, default=2)
    ap.add_argument("--premapped", action="store_true",
                    help="columns given as ids (mapping skipped, dim3_partition_ids); ids made on the host before timing")
    ap.add_argument("--cache-budget", type=int, default=None,
                    help="partial result cache of this many entries (Section 3), built before timing")
    ap.add_argument("--aggregate", default=None,
                    help="AGG:FN, e.g. sum:mul: time the Join-Aggregate (Section 4.1) on the workload, "
                         "values uniform in [-100, 100)")
    ap.add_argument("--mjp", type=int, default=0,
                    help="k: time the k-hop line query Pi(E join ... join E) (Section 4.2) on the workload's "
                         "edges, with the DP's deduplication placement and the two baseline plans")
    ap.add_argument("--f1-sweep", action="store_true",
                    help="Section 2.6's f1 on 1M x 1M uniform tables over a range of N_Y: one JSON line per "
                         "point with the forced hybrid and classical times and f1's choice")
    ap.add_argument("--count", action="store_true",
                    help="time dim3_join_count (Join-Aggregate COUNT per pair) instead of dim3_join_project")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (theta_z, DenseEC variant, emit rows) before timing")
    ap.add_argument("--no-sub", action="store_true",
                    help="default workload only: skip the batch256, serve2000 and chung_lu_1m_4m sub-records")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def make_workload(name: str, rank: int = 0, scale: float = 1.0):
    import gen

    if name == "two_table_1m_zipf1":
        return gen.config2_two_table(seed=1 + 1000 * rank, scale=scale)
    if name == "self_20k":
        return gen.config1_self(seed=0 + 1000 * rank)
    if name == "dense_16k":
        # DenseEC shape: |X| = |Y| = |Z| = 16384, 4M uniform tuples per table
        # (density 1.5%); with theta_z = 0 every z is dense and the tensor-core
        # product covers 2 * 16384^3 FLOP
        n = max(64, int(16384 * scale))
        return gen.two_table(np.random.default_rng(7 + 1000 * rank), 16 * n * n // 1024, 16 * n * n // 1024,
                             n, n, n, 0.0, name=f"dense_{n}")
    if name == "chung_lu_uncapped_x0.25":
        return gen.chung_lu_uncapped(seed=2 + 1000 * rank, scale=0.25 * scale)
    return gen.config3_chung_lu(seed=2 + 1000 * rank, scale=scale)


def premap(inst):
    """Rank ids of an instance's columns, as a database would hold them for
    auto-increment or dictionary-encoded columns: y over S.y (R tuples whose y
    is not in S.y get -1), x over R.x, z over S.z. Host numpy, outside any
    timed region."""
    yv, xv, zv = np.unique(inst.s_key), np.unique(inst.r_val), np.unique(inst.s_val)
    r_y = np.searchsorted(yv, inst.r_key)
    r_y = np.where((r_y < yv.size) & (yv[np.minimum(r_y, max(yv.size - 1, 0))] == inst.r_key), r_y, -1)
    cols = (r_y, np.searchsorted(xv, inst.r_val), np.searchsorted(yv, inst.s_key), np.searchsorted(zv, inst.s_val))
    return [np.ascontiguousarray(c, np.int32) for c in cols], (xv.size, yv.size, zv.size)


def measured_peaks():
    """HBM GB/s, bf16 TFLOP/s burst and sustained, and where they came from."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm": float(d["hbm_gbs"]), "bf16": float(d["bf16_tflops"]),
                "bf16_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "source": "measured"}
    except Exception:  # noqa: BLE001
        return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:  # noqa: BLE001
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(workload: str):
    """DRAM bytes per launch of the emitting kernel on `workload` from the
    committed ncu summary (scaled to the full launch), if it was taken on the
    current source of that kernel; else (None, entry or None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[workload]
        import hashlib

        src = os.path.join(ROOT, "paper_2206_04995_gb300", "csrc", e["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if h != e["source_sha"]:
            return None, e
        return float(e["dram_bytes_per_launch_full"]), e
    except Exception:  # noqa: BLE001
        return None, None


def reduce_over_ranks(dist, busy_s: float, pairs: int, device):
    """Whole-job numbers of N replicas: the slowest rank's busy time (max) and
    the pairs all ranks produced (sum). dist is torch.distributed or None."""
    if dist is None:
        return busy_s, float(pairs)
    import torch

    t = torch.tensor([busy_s, float(pairs)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


def rows_on_device(torch, out_x, out_z, xs: np.ndarray):
    """The (x, z) rows of a canonical device result whose x is in xs, as host
    arrays (searchsorted on the device, then one copy per row)."""
    xs = np.unique(np.asarray(xs, np.int32))
    q = torch.from_numpy(xs).to(out_x.device)
    lo = torch.searchsorted(out_x, q, right=False).cpu().numpy()
    hi = torch.searchsorted(out_x, q, right=True).cpu().numpy()
    px = [out_x[a:b].cpu().numpy() for a, b in zip(lo, hi) if b > a]
    pz = [out_z[a:b].cpu().numpy() for a, b in zip(lo, hi) if b > a]
    cat = (lambda p: np.concatenate(p) if p else np.zeros(0, np.int32))  # noqa: E731
    return cat(px), cat(pz)


def boundary_x(torch, out_x, total: int) -> np.ndarray:
    """x of the rows holding output positions 0, total - 1 and those next to
    2^31 and 2^32 (where 32-bit offsets would wrap)."""
    pos = sorted({p for p in [0, total - 1] + [b + d for b in (1 << 31, 1 << 32) for d in (-1, 0)]
                  if 0 <= p < total})
    if not pos:
        return np.zeros(0, np.int32)
    return np.unique(out_x[torch.tensor(pos, dtype=torch.int64, device=out_x.device)].cpu().numpy())


def cpu_baseline(inst, target_s: float, rng_seed: int = 5, check=None):
    """The oracle as it stands, single-threaded, on the rows of a random x
    sample sized to take about target_s seconds.

    ``check`` = (extra_x, rows_fn): the sample also holds the x values
    extra_x, and the oracle's rows are compared element by element with the
    GPU rows rows_fn(xs) of the timed output. Returns (baseline, verified)."""
    import oracle

    oracle.build()
    xs = np.unique(inst.r_val)
    extra = np.zeros(0, np.int32) if check is None else np.asarray(check[0], np.int32)
    rng = np.random.default_rng(rng_seed)
    k = 4
    while True:
        pick = np.unique(np.concatenate([rng.choice(xs, size=min(k, xs.size), replace=False), extra]))
        t0 = time.perf_counter()
        x, z, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val, x_filter=pick)
        dt = time.perf_counter() - t0
        if dt >= target_s * 0.5 or pick.size >= xs.size:
            break
        k = int(min(xs.size, max(k * 2, k * target_s / max(dt, 1e-3) * 0.9)))
    base = {"value": x.size / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"rows of {pick.size} x of {xs.size} (random, plus the first, the last and those holding "
                      f"output positions next to 2^31 and 2^32; R restricted to them, S whole); "
                      f"{x.size} pairs in {dt:.2f} s"}
    verified = None
    if check is not None:
        gx, gz = check[1](pick)
        ok = bool(gx.size == x.size and np.array_equal(gx, x) and np.array_equal(gz, z))
        verified = {"rows": int(pick.size), "pairs": int(x.size), "ok": ok,
                    "boundary_x": [int(v) for v in extra],
                    "how": "oracle rows (its x filter) vs the same rows of the last timed step's output, "
                           "element by element"}
    return base, verified


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    inst = make_workload(args.workload, 0, args.scale)
    import oracle

    oracle.build()
    xs = np.unique(inst.r_val)
    rng = np.random.default_rng(17)
    per_step = max(1, min(xs.size, 200))
    pairs = 0
    t_total = 0.0
    for s in range(args.warmup + args.steps):
        pick = rng.choice(xs, size=per_step, replace=False)
        t0 = time.perf_counter()
        x, _, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val, x_filter=pick)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            pairs += x.size
            t_total += dt
    value = pairs / t_total
    sample = f"each step: rows of {per_step} random x of {xs.size} (R restricted, S whole), single-threaded"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": inst.name},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    assert args.warmup >= 3 or os.environ.get("DIM3_BENCH_ALLOW_SHORT"), "at least 3 warm-up steps"
    if args.workload == "batch256":
        run_batch(args, rank, world, local_rank)
        return
    if args.workload == "serve2000":
        run_serve(args, rank, world, local_rank)
        return
    if args.aggregate:
        run_aggregate(args, rank, world, local_rank)
        return
    if args.mjp:
        run_mjp(args, rank, world, local_rank)
        return
    if args.f1_sweep:
        run_f1_sweep(args, local_rank)
        return

    import torch

    import paper_2206_04995_gb300 as dim3

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    inst = make_workload(args.workload, rank, args.scale)
    dev = torch.device("cuda", local_rank)
    host_cols = [inst.r_key, inst.r_val, inst.s_key, inst.s_val]
    ranges = None
    if args.premapped:
        host_cols, ranges = premap(inst)
    cols = device_columns(torch, host_cols, dev)
    ctx = dim3.Context(local_rank)
    dense_wl = args.workload.startswith("dense")
    theta = args.theta_z if args.theta_z is not None else (0 if dense_wl else None)
    variant = args.dense_variant if args.dense_variant is not None else (dim3.DENSE_TC if dense_wl else None)
    if theta is not None:
        ctx.set_option(dim3.OPT_THETA_Z, theta)
    if variant is not None:
        ctx.set_option(dim3.OPT_DENSE_VARIANT, variant)
    for kv in args.opt:
        k, v = kv.split("=")
        ctx.set_option(int(k), int(v))

    tuned = None
    if (not args.no_tune and theta is None and variant is None and not args.opt and ranges is None
            and args.cache_budget is None and not args.count):
        from paper_2206_04995_gb300 import tune

        tuned = tune.summary(tune.tune(ctx, cols, use_cache=False))

    cache = None
    cache_cfg = None
    if args.cache_budget is not None:
        assert ranges is None, "--cache-budget works on value columns"
        t0 = time.perf_counter()
        cache = ctx.cache_build(*cols, args.cache_budget)
        torch.cuda.synchronize()
        cache_cfg = dict(cache.info, budget=args.cache_budget, build_s=time.perf_counter() - t0,
                         t_sparse=dim3.Context.T_SPARSE, t_dense=dim3.Context.T_DENSE)

    def join_call(c, ox, oz):
        """The public path: one dim3_join_project; for pre-mapped ids
        dim3_partition_ids, for a cache dim3_partition_cached, each followed
        by dim3_plan_join_project + dim3_plan_destroy."""
        if ranges is None and cache is None:
            if args.count:
                return ctx.join_count(*c, out_x=ox, out_z=oz, out_c=out_c)[:2]
            return ctx.join_project(*c, out_x=ox, out_z=oz)
        pl = ctx.partition_cached(*c, cache) if cache is not None else ctx.partition_ids(*c, *ranges)
        try:
            return pl.join_project(out_x=ox, out_z=oz)
        finally:
            pl.close()

    # size the output once (plan path), then time the one-call path
    if cache is not None:
        plan = ctx.partition_cached(*cols, cache)
    else:
        plan = ctx.partition_ids(*cols, *ranges) if ranges else ctx.partition(*cols)
    info = plan.info
    out_p = int(plan.row_counts().sum().item())
    plan.close()
    out_x = torch.empty(out_p, dtype=torch.int32, device=dev)
    out_z = torch.empty(out_p, dtype=torch.int32, device=dev)
    out_c = torch.empty(out_p if args.count else 0, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > 129 MB L2

    def step():
        x, _ = join_call(cols, out_x, out_z)
        return x.numel()

    for _ in range(args.warmup):
        assert step() == out_p
    torch.cuda.synchronize()

    ctx.set_option(dim3.OPT_TIMING, 1)
    ctx.timing(reset=True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = dim3.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    evs = []
    for k in range(args.steps):
        flush.fill_(k)  # evict the previous step's lines from L2 (outside the step's events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        n = step()
        e1.record()
        evs.append((e0, e1))
        assert n == out_p
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    launches = dim3.launch_count() - l0
    clocks = sampler.stop()
    tm = ctx.timing()
    ctx.set_option(dim3.OPT_TIMING, 0)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    busy_s = sum(step_ms) / 1e3

    total_pairs = out_p * args.steps
    busy_max, pairs_all = reduce_over_ranks(dist, busy_s, total_pairs, dev)
    value = pairs_all / busy_max

    # roofline of the dominant kernel: SparseBMM + union + compaction (emitting
    # pass, HBM-bound), or the tensor-core DenseEC product when every z is dense
    peaks = measured_peaks()
    # per-step totals (a phase may hold several launches per step, e.g. the
    # bitmap rows and the light rows of one pass)
    phases = {k: round(v[0] / args.steps, 4) for k, v in tm.items() if v[1]}
    tc_ms, tc_n = tm["dense_tc"]
    if tc_n and tc_ms > tm["sparse_emit"][0]:
        tc_s = tc_ms / 1e3 / tc_n
        flops = 2.0 * info["n_x"] * info["n_y_dense"] * info["n_z_dense"]
        peak = peaks["bf16"] * FP8_PER_BF16
        achieved = flops / tc_s / 1e12
        roofline = {"bound": "tensor", "kernel": "k_dense_tc (tcgen05 kind::f8f6f4, 0/1 operands)",
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_source": f"{peaks['source']} bf16 burst x {FP8_PER_BF16} (fp8/bf16 nominal ratio)",
                    "traffic": None, "alg_flops_per_launch": flops, "launch_ms": tc_s * 1e3}
    else:
        emit_ms, emit_n = tm["sparse_emit"]
        emit_s = emit_ms / 1e3 / args.steps  # the whole emitting pass of one step
        alg_bytes = (12 if args.count else 8) * out_p + 4 * info["n_r_kept"] + 4 * info["n_s_sparse"]
        achieved = alg_bytes / emit_s / 1e9
        traffic, tinfo = traffic_for(args.workload) if not args.count else (None, {"kernel": "k_xrow_counts<emit>"})
        tiled = args.workload == "chung_lu_1m_4m" and not args.count
        kname = (tinfo or {}).get("kernel", "k_place_rows (rows staged by k_tiled_rows<stage> + k_light_rows<stage>)"
                                  if tiled else "k_xrow_emit_g / k_xrow_bits<emit>")
        roofline = {"bound": "hbm", "kernel": f"{kname} (SparseBMM+union+compaction)",
                    "achieved": achieved, "peak": peaks["hbm"], "unit": "GB/s", "frac": achieved / peaks["hbm"],
                    "peak_source": peaks["source"], "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                    "launch_ms": emit_s * 1e3}

    e2e = None
    if not args.no_e2e and args.e2e_steps > 0 and not args.count:
        e2e = run_e2e(torch, host_cols, join_call, dev, out_p, args.e2e_steps)

    cpu, verified = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's sample also checks the timed output: its rows are
        # compared with the same rows of the last timed step
        check = None
        if cache is None and ranges is None and not args.count:
            check = (boundary_x(torch, out_x, out_p), lambda xs: rows_on_device(torch, out_x, out_z, xs))
        cpu, verified = cpu_baseline(inst, args.cpu_seconds, check=check)

    sub = None
    if (rank == 0 and world == 1 and not args.no_sub and args.workload == "two_table_1m_zipf1" and args.scale == 1.0
            and ranges is None and cache is None and not args.count):
        # the other configured workloads, each with its own timing: the
        # headline's buffers are released first
        ctx.close()
        del out_x, out_z, out_c, flush
        torch.cuda.empty_cache()
        sub = {"batch256": run_batch(args, rank, world, local_rank, sub=True),
               "chung_lu_1m_4m": onecall_record("chung_lu_1m_4m", local_rank),
               "chung_lu_uncapped_x0.25": onecall_record("chung_lu_uncapped_x0.25", local_rank),
               "dense_16k": onecall_record("dense_16k", local_rank),
               # every z dense on the tensor cores (the tuner's choice above is
               # all sparse on GB300): DenseEC's own roofline, same exact result
               "dense_16k_tc": onecall_record("dense_16k", local_rank, tune_it=False,
                                              opts={dim3.OPT_THETA_Z: 0, dim3.OPT_DENSE_VARIANT: dim3.DENSE_TC}),
               "serve2000": serve_record(args, local_rank)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * busy_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": inst.name + (" (Join-Count)" if args.count else ""), "n_r": inst.nr, "n_s": inst.ns, "n_x": info["n_x"],
                       "n_y": info["n_y"], "n_z": info["n_z"], "n_z_dense": info["n_z_dense"],
                       "out_p": out_p, "out_j": info["out_j"], "theta_z": info["theta_z"],
                       "l2": "flushed between steps (256 MiB write outside the step events)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "mapping": ("skipped: pre-mapped id columns (dim3_partition_ids); output pairs are ids"
                                   if ranges else "order-preserving hash + radix rank (dim3_join_project)"),
                       "partial_result_cache": cache_cfg, "tuner": tuned,
                       "join_tuples_per_s": info["out_j"] * args.steps * (pairs_all / total_pairs) / busy_max},
            "roofline": roofline,
            "phase_ms": phases,
            "partition_roofline": partition_roofline(info, phases, peaks["hbm"]),
            "sparse_roofline": (sparse_passes_roofline(tm, args.steps, roofline["alg_bytes_per_launch"], peaks)
                                if roofline["bound"] == "hbm" else None),
            "wall_s": t_wall,
            "gpu_launches": launches,
            "clocks": clocks,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "verified": verified,
            "sub": sub,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    ctx.close()


def partition_roofline(info: dict, phase_ms: dict, peak_gbs: float) -> dict:
    """Mapping + partition (a2-a6) against HBM: algorithmic bytes per call =
    16 B per input tuple (key and value read, two ids written), 4 B per
    dictionary entry, 12 B per R' and S tuple for the CSRs (8 B read, 4 B
    column written), 8 B per row pointer; over the phases' device time."""
    alg = (16 * (info["n_r"] + info["n_s"]) + 4 * (info["n_x"] + info["n_y"] + info["n_z"]) +
           12 * (info["n_r_kept"] + info["n_s"]) + 8 * (info["n_x"] + info["n_y"] + 2))
    ms = phase_ms.get("map", 0.0) + phase_ms.get("partition", 0.0)
    gbs = alg / (ms / 1e3) / 1e9 if ms > 0 else None
    return {"alg_bytes": alg, "ms": ms, "achieved_gbs": gbs, "frac": gbs / peak_gbs if gbs else None}


def onecall_record(name: str, local_rank: int, steps: int = 5, warmup: int = 3, tune_it: bool = True,
                   opts: dict | None = None):
    """A compact record of one workload through the one-call path
    (dim3_join_project into caller buffers), tuned first (or with the given
    context options instead): pairs/s, phases and the emitting pass's HBM
    roofline (and the tensor-core DenseEC's when it ran)."""
    import torch

    import paper_2206_04995_gb300 as dim3

    dev = torch.device("cuda", local_rank)
    inst = make_workload(name, 0)
    cols = device_columns(torch, [inst.r_key, inst.r_val, inst.s_key, inst.s_val], dev)
    ctx = dim3.Context(local_rank)
    tuned = None
    for k, v in (opts or {}).items():
        ctx.set_option(k, v)
    if tune_it and not opts:
        from paper_2206_04995_gb300 import tune

        tuned = tune.summary(tune.tune(ctx, cols, use_cache=False))
    plan = ctx.partition(*cols)
    info = plan.info
    out_p = int(plan.row_counts().sum().item())
    plan.close()
    out_x = torch.empty(out_p, dtype=torch.int32, device=dev)
    out_z = torch.empty(out_p, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    for _ in range(warmup):
        ctx.join_project(*cols, out_x=out_x, out_z=out_z)
    torch.cuda.synchronize()
    ctx.set_option(dim3.OPT_TIMING, 1)
    ctx.timing(reset=True)
    ms = []
    for k in range(steps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, _ = ctx.join_project(*cols, out_x=out_x, out_z=out_z)
        e1.record()
        torch.cuda.synchronize()
        assert x.numel() == out_p
        ms.append(e0.elapsed_time(e1))
    tm = ctx.timing()
    ctx.close()
    peaks = measured_peaks()
    dense = None
    if tm["dense_tc"][1]:
        tc_s = tm["dense_tc"][0] / 1e3 / tm["dense_tc"][1]
        flops = 2.0 * info["n_x"] * info["n_y_dense"] * info["n_z_dense"]
        peak = peaks["bf16"] * FP8_PER_BF16
        dense = {"bound": "tensor", "kernel": "k_dense_tc", "achieved": flops / tc_s / 1e12, "peak": peak,
                 "unit": "TFLOP/s", "frac": flops / tc_s / 1e12 / peak, "launch_ms": tc_s * 1e3,
                 "peak_source": f"{peaks['source']} bf16 burst x {FP8_PER_BF16} (fp8/bf16 nominal ratio)"}
    emit_s = tm["sparse_emit"][0] / 1e3 / steps
    alg_bytes = 8 * out_p + 4 * info["n_r_kept"] + 4 * info["n_s_sparse"]
    achieved = alg_bytes / emit_s / 1e9 if emit_s > 0 else None
    del out_x, out_z, flush
    torch.cuda.empty_cache()
    return {"pairs_per_s": out_p * steps / (sum(ms) / 1e3), "ms_per_step": sum(ms) / steps, "steps": steps,
            "out_p": out_p, "out_j": info["out_j"], "n_x": info["n_x"], "n_z": info["n_z"],
            "n_z_dense": info["n_z_dense"], "phase_ms": {k: round(v[0] / steps, 4) for k, v in tm.items() if v[1]},
            "roofline": {"bound": "hbm", "kernel": "emitting pass (k_place_rows after staging, or k_tiled_rows<emit> "
                         "+ k_light_rows<emit>, or k_xrow_emit_g)", "achieved": achieved, "peak": peaks["hbm"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm"] if achieved else None, "peak_source": peaks["source"],
                         "alg_bytes_per_launch": alg_bytes, "launch_ms": emit_s * 1e3},
            # the whole SparseBMM + compaction (counting or staging pass plus
            # emitting pass) against the same algorithmic bytes
            "sparse_roofline": sparse_passes_roofline(tm, steps, alg_bytes, peaks),
            "dense_roofline": dense,
            "partition_roofline": partition_roofline(info, {k: v[0] / steps for k, v in tm.items() if v[1]},
                                                     peaks["hbm"]),
            "tuner": tuned, "l2": "flushed between steps"}


def sparse_passes_roofline(tm, steps: int, alg_bytes: float, peaks):
    """HBM fraction of both SparseBMM passes together (counting or staging
    pass + emitting pass), per step."""
    ms = (tm["sparse_count"][0] + tm["sparse_emit"][0]) / steps
    if ms <= 0:
        return None
    gbs = alg_bytes / (ms / 1e3) / 1e9
    return {"kernels": "k_tiled_rows<stage> + k_light_rows<stage> + k_place_rows, or count + emit",
            "alg_bytes": alg_bytes, "ms": ms, "achieved_gbs": gbs, "frac": gbs / peaks["hbm"]}


def serve_record(args, local_rank: int):
    """A compact record of the full query stream, served and plain, queued
    and Poisson (see run_serve)."""
    import torch

    dev = torch.device("cuda", local_rank)
    t0 = time.perf_counter()
    qs = serve_queries(torch, args.serve_queries, args.serve_max_tuples, 0, dev)
    gen_s = time.perf_counter() - t0
    serve_runs(torch, qs[: min(len(qs), 40)], local_rank, args.serve_workers, modes=("queued",))
    r = serve_runs(torch, qs, local_rank, args.serve_workers)
    keep = ("pairs_per_s", "wall_s", "p50_ms", "p99_ms", "mean_batch", "offered_pairs_per_s")
    out = {k: ({kk: v[kk] for kk in keep} if isinstance(v, dict) else v) for k, v in r.items()}
    out.update(queries=len(qs), pairs=r["served_queued"]["pairs"], tuples=int(sum(q.tuples for q in qs)),
               inputs_s=gen_s, workers=args.serve_workers)
    del qs
    torch.cuda.empty_cache()
    return out


def run_batch(args, rank, world, local_rank, sub=False):
    """256 independent two-table instances (log-uniform sizes): one step is
    ONE dim3_batch_join_project call over all of them; the same instances run
    one call each (the plain path) beside it for the ratio. With sub, returns
    a compact record (no end-to-end or oracle legs) instead of printing."""
    import torch

    import gen
    import paper_2206_04995_gb300 as dim3

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    insts = gen.config4_batch(seed=3 + 1000 * rank, n_inst=args.batch_insts)
    cols = [[torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(dev)
             for a in (i.r_key, i.r_val, i.s_key, i.s_val)] for i in insts]
    ctx = dim3.Context(local_rank)
    for kv in args.opt:
        k, v = kv.split("=")
        ctx.set_option(int(k), int(v))
    tuned = None
    if not args.no_tune and not args.opt:
        from paper_2206_04995_gb300 import tune

        tuned = tune.summary(tune.tune(ctx, cols, batch=True, use_cache=False))
    steps, warmup = (10, 3) if sub else (args.steps, args.warmup)
    plan = ctx.batch_partition(cols)
    info = plan.info
    out_p = int(plan.row_counts().sum().item())
    plan.close()
    out_x = torch.empty(out_p, dtype=torch.int32, device=dev)
    out_z = torch.empty(out_p, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def batched():
        x, _, _ = ctx.batch_join_project(cols, out_x=out_x, out_z=out_z)
        return x.numel()

    # the plain path: one dim3_join_project per instance into the same buffers
    sizes = []
    for c in cols:
        p = ctx.partition(*c)
        sizes.append(int(p.row_counts().sum().item()))
        p.close()
    offs = np.concatenate([[0], np.cumsum(sizes)])

    def plain():
        n = 0
        for t, c in enumerate(cols):
            x, _ = ctx.join_project(*c, out_x=out_x[offs[t]:offs[t + 1]], out_z=out_z[offs[t]:offs[t + 1]])
            n += x.numel()
        return n

    def timed(fn, steps):
        ms = []
        for k in range(steps):
            flush.fill_(k)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            assert fn() == out_p
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    for _ in range(warmup):
        batched()
        plain()
    torch.cuda.synchronize()
    plain_ms = timed(plain, max(1, min(steps, 3)))
    ctx.set_option(dim3.OPT_TIMING, 1)
    ctx.timing(reset=True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = dim3.launch_count()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    batch_ms = timed(batched, steps)
    t_wall = time.perf_counter() - t_wall
    launches = dim3.launch_count() - l0
    clocks = sampler.stop()
    tm = ctx.timing()
    ctx.set_option(dim3.OPT_TIMING, 0)
    busy = sum(batch_ms) / 1e3
    value = out_p * steps / busy
    plain_value = out_p * len(plain_ms) / (sum(plain_ms) / 1e3)
    peaks = measured_peaks()
    emit_ms, emit_n = tm["sparse_emit"]
    emit_s = emit_ms / 1e3 / max(emit_n, 1)
    alg_bytes = 8 * out_p + 4 * info["n_r_kept"] + 4 * info["n_s_sparse"]
    achieved = alg_bytes / emit_s / 1e9
    # the emitting kernel over all instances: k_xrow_emit_g<G> with G rows of
    # one instance per CTA (the tuner's choice), or k_xrow_bits<emit> with one
    G = (tuned or {}).get("emit_rows") or next((int(kv.split("=")[1]) for kv in args.opt if kv.split("=")[0] == "6"), 0) or 2
    kname = f"k_xrow_emit_g<{G}> over all instances" if G > 1 else "k_xrow_bits<emit> over all instances"
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved,
                "peak": peaks["hbm"], "unit": "GB/s", "frac": achieved / peaks["hbm"],
                "peak_source": peaks["source"], "traffic": None, "alg_bytes_per_launch": alg_bytes,
                "launch_ms": emit_s * 1e3}
    phase_ms = {k: round(v[0] / max(v[1], 1), 4) for k, v in tm.items() if v[1]}
    if sub:
        ctx.close()
        return {"pairs_per_s": value, "ms_per_step": sum(batch_ms) / len(batch_ms), "steps": steps,
                "plain_pairs_per_s": plain_value, "plain_ms_per_step": sum(plain_ms) / len(plain_ms),
                "batched_over_plain": value / plain_value, "out_p": out_p, "n_inst": len(insts),
                "roofline": roofline, "phase_ms": phase_ms, "gpu_launches": launches, "tuner": tuned,
                "partition_roofline": partition_roofline(info, phase_ms, peaks["hbm"])}
    e2e = None
    if not args.no_e2e:
        h_in = [[c.cpu().pin_memory() for c in cc] for cc in cols]
        h_x = torch.empty(out_p, dtype=torch.int32, pin_memory=True)
        h_z = torch.empty(out_p, dtype=torch.int32, pin_memory=True)

        def e2e_step():
            for d, h in zip(cols, h_in):
                for dd, hh in zip(d, h):
                    dd.copy_(hh, non_blocking=True)
            x, z, _ = ctx.batch_join_project(cols, out_x=out_x, out_z=out_z)
            h_x.copy_(x, non_blocking=True)
            h_z.copy_(z, non_blocking=True)
            return x.numel()

        e2e_ms = timed(e2e_step, max(1, min(args.steps, args.e2e_steps)))
        e2e = {"value": out_p * len(e2e_ms) / (sum(e2e_ms) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": sum(i.nr + i.ns for i in insts) * 8, "d2h_bytes_per_step": 8 * out_p,
               "host_memory": "pinned", "ms_per_step": sum(e2e_ms) / len(e2e_ms)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        small = sorted(insts, key=lambda i: i.nr)[:: max(1, len(insts) // 16)][:16]
        import oracle

        oracle.build()
        t0 = time.perf_counter()
        n = sum(oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)[0].size for i in small)
        dt = time.perf_counter() - t0
        cpu = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{len(small)} of the 256 instances (every 16th by size), whole; {n} pairs in {dt:.2f} s"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": sum(batch_ms) / len(batch_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "batch256", "n_inst": len(insts), "tuples": int(sum(i.nr + i.ns for i in insts)),
                       "out_p": out_p, "out_j": info["out_j"], "plain_pairs_per_s": plain_value,
                       "plain_ms_per_step": sum(plain_ms) / len(plain_ms), "batched_over_plain": value / plain_value,
                       "tuner": tuned, "l2": "flushed between steps (256 MiB write outside the step events)"},
            "roofline": roofline,
            "phase_ms": phase_ms,
            "wall_s": t_wall, "gpu_launches": launches, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu,
        }), flush=True)
    ctx.close()


def serve_queries(torch, n_queries: int, hi: int, rank: int, dev):
    """The Poisson stream of Join-Project / Join-Count queries (arrivals,
    kinds, sizes and seeds from gen.config5_stream), each query's tables drawn
    on the device from its seed (gen.device) and kept in page-locked host
    memory, from where the server copies them in."""
    import gen
    from gen import device as gdev
    from paper_2206_04995_gb300.serve import Query

    stream = gen.config5_stream(seed=4 + 1000 * rank, n_queries=n_queries, hi=hi)
    qs = []
    for i, q in enumerate(stream):
        cols = [c.cpu().pin_memory() for c in gdev.query_tables(q, dev)]
        qs.append(Query(i, q.kind, *cols, q.arrival_s))
    torch.cuda.synchronize()
    return qs


def serve_runs(torch, qs, local_rank, workers: int, modes=("queued", "poisson")):
    """Served (continuous batching, `workers` streams) and plain (one query at
    a time on one stream, every query alone) runs of the stream: all queued at
    once (capacity) and arriving at their Poisson times (latency). Results are
    handed over in chunks and released at once (the consumer only counts)."""
    import dataclasses

    from paper_2206_04995_gb300.serve import Limits, Server, summarize

    served_lim = Limits(max_batch=64, max_tuples=16_000_000, reserve_bytes=8 << 30)
    plain_lim = Limits(max_batch=1, reserve_bytes=8 << 30, big_tuples=0)
    out = {}
    for mode in modes:
        for name, w, lim in (("served", workers, served_lim), ("plain", 1, plain_lim)):
            srv = Server(local_rank, workers=w, limits=lim, keep=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = srv.run([dataclasses.replace(q) for q in qs], realtime=(mode == "poisson"))
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            srv.close()
            sm = summarize(res, wall)
            span = max(q.arrival for q in qs) if mode == "poisson" else 0.0
            sm["offered_pairs_per_s"] = sm["pairs"] / span if span > 0 else None
            out[f"{name}_{mode}"] = sm
            torch.cuda.empty_cache()
    for mode in modes:
        out[f"served_over_plain_{mode}"] = out[f"served_{mode}"]["pairs_per_s"] / out[f"plain_{mode}"]["pairs_per_s"]
    return out


def run_serve(args, rank, world, local_rank):
    """The Poisson query stream (2,000 queries at 200 q/s, tuples log-uniform
    in [1e4, 2e6] per table, half Join-Project and half Join-Count): served
    by the continuous-batching loop and by the plain loop, all queued at once
    and arriving at their Poisson times."""
    import torch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t0 = time.perf_counter()
    qs = serve_queries(torch, args.serve_queries, args.serve_max_tuples, rank, dev)
    gen_s = time.perf_counter() - t0
    # warm-up: contexts, module loading, memory pools
    serve_runs(torch, qs[: min(len(qs), 40)], local_rank, args.serve_workers, modes=("queued",))
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = dim3_launch_count()
    r = serve_runs(torch, qs, local_rank, args.serve_workers)
    launches = dim3_launch_count() - l0
    clocks = sampler.stop()
    cap = r["served_queued"]
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": cap["pairs_per_s"], "unit": UNIT, "n_gpus": world, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * cap["wall_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "serve2000", "queries": len(qs), "max_tuples": args.serve_max_tuples,
                       "rate_qps": 200.0, "workers": args.serve_workers, "inputs_s": gen_s,
                       "tuples": int(sum(q.tuples for q in qs)), **r,
                       "p50_ms": r["served_poisson"]["p50_ms"], "p99_ms": r["served_poisson"]["p99_ms"]},
            "gpu_launches": launches, "clocks": clocks,
            "e2e": {"value": cap["pairs_per_s"], "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(q.tuples for q in qs) * 8), "d2h_bytes_per_step": 0,
                    "note": "inputs copied in from page-locked host memory per query; results stay on the "
                            "device, handed to the consumer chunk by chunk and released"},
        }), flush=True)


def dim3_launch_count():
    import paper_2206_04995_gb300 as dim3

    return dim3.launch_count()


def run_aggregate(args, rank, world, local_rank):
    """Join-Aggregate G_{x,z} agg(f(R.v, S.u)) on the workload's tables with
    seeded values: groups per second, one dim3_join_aggregate per step into
    preallocated buffers (mapping, partition, counting pass, per-pair value
    statistics, aggregate SPA pass)."""
    import torch

    import paper_2206_04995_gb300 as dim3

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    agg_name, fn_name = args.aggregate.split(":")
    agg = {"count": dim3.AGG_COUNT, "sum": dim3.AGG_SUM, "min": dim3.AGG_MIN, "max": dim3.AGG_MAX,
           "avg": dim3.AGG_AVG}[agg_name]
    fn = {"mul": dim3.FN_MUL, "add": dim3.FN_ADD, "left": dim3.FN_LEFT, "right": dim3.FN_RIGHT}[fn_name]
    inst = make_workload(args.workload, rank, args.scale)
    rng = np.random.default_rng(17 + rank)
    r_v = rng.integers(-100, 100, inst.r_key.size).astype(np.int32)
    s_u = rng.integers(-100, 100, inst.s_key.size).astype(np.int32)
    cols = [torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(dev)
            for a in (inst.r_key, inst.r_val, r_v, inst.s_key, inst.s_val, s_u)]
    ctx = dim3.Context(local_rank)
    x, z, v = ctx.join_aggregate(*cols, agg, fn)
    n = x.numel()
    out = (x, z, v)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        ctx.join_aggregate(*cols, agg, fn, out=out)
    torch.cuda.synchronize()
    ctx.set_option(dim3.OPT_TIMING, 1)
    ctx.timing(reset=True)
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = dim3.launch_count()
    ms = []
    for k in range(args.steps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.join_aggregate(*cols, agg, fn, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    launches = dim3.launch_count() - l0
    tm = ctx.timing()
    busy = sum(ms) / 1e3
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n * args.steps / busy, "unit": "groups/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * busy / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": inst.name, "aggregate": args.aggregate, "groups": n, "n_r": inst.nr,
                       "n_s": inst.ns, "l2": "flushed between steps (256 MiB write outside the step events)"},
            "phase_ms": {k: round(a / max(b, 1), 4) for k, (a, b) in tm.items() if b},
            "gpu_launches": launches, "clocks": clocks,
        }), flush=True)
    ctx.close()


def run_mjp(args, rank, world, local_rank):
    """k-hop line query over the workload's R as an edge list (x -> y):
    exact chain sizes, the DP's deduplication placement (Section 4.2), and
    the time of that plan against deduplicating after every join and only
    after the last (skipped when its bag would not fit in memory). Result
    pairs per second of the DP's plan."""
    import torch

    import paper_2206_04995_gb300 as dim3

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    inst = make_workload(args.workload, rank, args.scale)
    a = torch.from_numpy(np.ascontiguousarray(inst.r_val, np.int32)).to(dev)
    b = torch.from_numpy(np.ascontiguousarray(inst.r_key, np.int32)).to(dev)
    k = args.mjp
    tables = [(a, b)] * k
    ctx = dim3.Context(local_rank)
    t0 = time.perf_counter()
    out_j, out_p = ctx.mjp_sizes(tables)
    sizes_s = time.perf_counter() - t0
    n_edges = float(np.unique(np.stack([inst.r_val, inst.r_key], 1), axis=0).shape[0])
    dedup, est = dim3.Context.mjp_plan([n_edges] * k, out_j, out_p)
    n = int(out_p[-1])
    out = (torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.int32, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    def timed(flags):
        for _ in range(args.warmup):
            ctx.mjp_execute(tables, flags, out=out)
        torch.cuda.synchronize()
        ms = []
        for i in range(args.steps):
            flush.fill_(i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x, _ = ctx.mjp_execute(tables, flags, out=out)
            e1.record()
            torch.cuda.synchronize()
            assert x.numel() == n
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = dim3.launch_count()
    dp_ms = timed(dedup)
    launches = dim3.launch_count() - l0
    clocks = sampler.stop()
    plans = {"dp": {"dedup": dedup, "ms": dp_ms, "estimate": est}}
    every = [False] + [True] * (k - 1)
    plans["every_join"] = {"dedup": every, "ms": dp_ms if every == dedup else timed(every)}
    last = [False] * (k - 1) + [True]
    bag = max(out_j[:-1]) if k > 1 else 0.0
    if bag * 16 < 0.5 * torch.cuda.get_device_properties(dev).total_memory:
        plans["last_only"] = {"dedup": last, "ms": dp_ms if last == dedup else timed(last)}
    else:
        plans["last_only"] = {"dedup": last, "ms": None, "skipped": f"bag of {bag:.3g} pairs"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n / (dp_ms / 1e3), "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dp_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{inst.name} {k}-hop line query", "edges": n_edges, "out_j": out_j,
                       "out_p": out_p, "sizes_s": sizes_s, "plans": plans,
                       "l2": "flushed between steps (256 MiB write outside the step events)"},
            "gpu_launches": launches, "clocks": clocks,
        }), flush=True)
    ctx.close()


def run_f1_sweep(args, local_rank):
    """f1 (Section 2.6) against measurement: |R| = |S| = 1e6 tuples, x and z
    uniform over [-1e8, 1e8), y uniform over [0, N_Y); for each N_Y one
    dim3_join_project into caller-sized buffers, best of `--steps` calls
    after `--warmup`, with the path forced hybrid, forced classical, and left
    to f1 (default constants). Prints one JSON line per N_Y."""
    import torch

    import paper_2206_04995_gb300 as dim3

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(local_rank)
    n = 1_000_000
    for ny in (3 * 10**3, 10**4, 3 * 10**4, 10**5, 3 * 10**5, 10**6, 10**7, 10**8):
        rng = np.random.default_rng(0)
        cols = [torch.from_numpy(a.astype(np.int32)).to(dev) for a in
                (rng.integers(0, ny, n), rng.integers(-10**8, 10**8, n), rng.integers(0, ny, n),
                 rng.integers(-10**8, 10**8, n))]
        ctx = dim3.Context(local_rank)
        plan = ctx.partition(*cols)
        out_j = int(plan.info["out_j"])
        out_p = int(plan.row_counts().sum().item())
        plan.close()
        ox = torch.empty(max(out_p, 1), dtype=torch.int32, device=dev)
        oz = torch.empty_like(ox)
        line = {"n_r": n, "n_s": n, "n_y": ny, "out_j": out_j, "out_p": out_p}
        for path, name in ((dim3.PATH_HYBRID, "hybrid_ms"), (dim3.PATH_CLASSICAL, "classical_ms"),
                           (dim3.PATH_AUTO, "f1_ms")):
            ctx.set_option(dim3.OPT_PATH, path)
            for _ in range(args.warmup):
                ctx.join_project(*cols, out_x=ox, out_z=oz)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(max(args.steps, 1)):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                x, _ = ctx.join_project(*cols, out_x=ox, out_z=oz)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
                assert x.numel() == out_p
            line[name] = round(best, 4)
            if path == dim3.PATH_AUTO:
                line["f1_chose"] = "hybrid" if ctx.last_path() == 1 else "classical"
        print(json.dumps(line), flush=True)
        ctx.close()
        del ox, oz
        torch.cuda.empty_cache()


def device_columns(torch, host_cols, dev):
    """Device copies of the host columns; a column given twice (a self-join's
    R and S) is copied once and passed twice, which the library detects as a
    self-join and maps once."""
    seen = {}
    out = []
    for a in host_cols:
        if id(a) not in seen:
            seen[id(a)] = torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(dev)
        out.append(seen[id(a)])
    return out


def gpu_numa(torch, dev) -> dict:
    """The GPU's PCI address and what sysfs says of its NUMA placement: its
    node and the CPUs local to it, with the node those CPUs belong to."""
    out = {"pci": None, "numa_node": None, "local_cpus": None, "cpu_node": None}
    try:
        pr = torch.cuda.get_device_properties(dev)
        pci = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        out["pci"] = pci
        base = f"/sys/bus/pci/devices/{pci}"
        with open(base + "/numa_node") as f:
            out["numa_node"] = int(f.read().strip())
        with open(base + "/local_cpulist") as f:
            out["local_cpus"] = f.read().strip()
        first = int(out["local_cpus"].split(",")[0].split("-")[0])
        import glob

        for nd in glob.glob("/sys/devices/system/node/node*/cpu%d" % first):
            out["cpu_node"] = int(nd.split("/node")[-1].split("/")[0].replace("node", ""))
    except Exception:  # noqa: BLE001
        pass
    return out


def host_region_info(addr: int) -> dict:
    """Where the pages of the mapping holding host address addr live: pages per
    NUMA node (/proc/self/numa_maps) and the bytes on transparent huge pages
    (AnonHugePages of /proc/self/smaps)."""
    out = {"numa_pages": None, "anon_huge_bytes": None}
    try:
        start = None
        with open("/proc/self/smaps") as f:
            cur = None
            for line in f:
                head = line.split()[0]
                if "-" in head and ":" not in head:
                    lo, hi = (int(v, 16) for v in head.split("-"))
                    cur = lo if lo <= addr < hi else None
                    if cur is not None:
                        start = cur
                elif cur is not None and line.startswith("AnonHugePages:"):
                    out["anon_huge_bytes"] = int(line.split()[1]) * 1024
        if start is not None:
            with open("/proc/self/numa_maps") as f:
                for line in f:
                    parts = line.split()
                    if int(parts[0], 16) == start:
                        out["numa_pages"] = {p.split("=")[0]: int(p.split("=")[1]) for p in parts
                                             if p[:1] == "N" and "=" in p}
                        break
    except Exception:  # noqa: BLE001
        pass
    return out


def bind_to_node(addr: int, nbytes: int, node: int) -> bool:
    """mbind(MPOL_BIND) of [addr, addr + nbytes) to one NUMA node, before its
    pages are touched (Linux syscall, x86_64 and aarch64 numbers)."""
    import ctypes
    import platform

    nr = {"x86_64": 237, "aarch64": 235}.get(platform.machine())
    if nr is None or node is None or node < 0 or node >= 64:
        return False
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        mask = ctypes.c_ulong(1 << node)
        rc = libc.syscall(ctypes.c_long(nr), ctypes.c_void_p(addr), ctypes.c_ulong(nbytes), ctypes.c_int(2),
                          ctypes.byref(mask), ctypes.c_ulong(64), ctypes.c_uint(0))
        return rc == 0
    except Exception:  # noqa: BLE001
        return False


def pinned_host_empty(torch, n, node=None):
    """(tensor, release, info) for an int32 CPU tensor of n elements in
    page-locked memory on transparent huge pages (anonymous mmap +
    MADV_HUGEPAGE, bound to NUMA node `node` when given, then
    cudaHostRegister), on which large device-to-host copies run at link speed
    consistently; release() undoes the registration; info says where the
    pages landed. The fallback is torch's pinned allocator (release None)."""
    import mmap

    try:
        nbytes = max(n, 1) * 4
        m = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        if hasattr(mmap, "MADV_HUGEPAGE"):
            m.madvise(mmap.MADV_HUGEPAGE)
        a = np.frombuffer(m, dtype=np.int32, count=max(n, 1))
        bound = bind_to_node(a.ctypes.data, nbytes, node) if node is not None else False
        for o in range(0, a.size, 1 << 26):  # fault the pages in (huge pages where the kernel has them)
            a[o:o + (1 << 26)] = 0
        rt = torch.cuda.cudart()
        r = rt.cudaHostRegister(a.ctypes.data, nbytes, 0)
        if getattr(r, "value", r) != 0:
            raise RuntimeError(f"cudaHostRegister: {r}")
        t = torch.from_numpy(a)[:n]

        def release():
            rt.cudaHostUnregister(a.ctypes.data)

        return t, release, dict(host_region_info(a.ctypes.data), bound_node=node if bound else None)
    except Exception:  # noqa: BLE001
        return torch.empty(n, dtype=torch.int32, pin_memory=True), None, None


def run_e2e(torch, host_cols, join_call, dev, out_p, steps):
    """Same metric through the public call with HOST buffers: pinned host
    inputs copied in, the join (``join_call``), both output columns copied out
    (side by side on two streams when the host columns are page-locked).
    The output columns are placed on the NUMA node of the CPUs local to the
    GPU when sysfs names one. A further, separately timed step records each
    copy's time and rate, and the record says where the host pages landed."""
    pin = True
    # a column given twice (a self-join's R and S) is copied once
    uniq, idx = [], []
    for a in host_cols:
        k = next((i for i, u in enumerate(uniq) if u is a), None)
        if k is None:
            uniq.append(a)
            k = len(uniq) - 1
        idx.append(k)
    releases, placement = [], []
    gpu = gpu_numa(torch, dev)
    try:
        h_in = [torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory() for a in uniq]
        (h_x, rx, ix), (h_z, rz, iz) = (pinned_host_empty(torch, out_p, gpu["cpu_node"]),
                                        pinned_host_empty(torch, out_p, gpu["cpu_node"]))
        releases = [r for r in (rx, rz) if r is not None]
        placement = [ix, iz]
        pin = h_x.is_pinned() and h_z.is_pinned()
    except Exception:  # noqa: BLE001
        pin = False
        h_in = [torch.from_numpy(np.ascontiguousarray(a, np.int32)) for a in uniq]
        h_x = torch.empty(out_p, dtype=torch.int32)
        h_z = torch.empty(out_p, dtype=torch.int32)
    d_in = [torch.empty_like(h, device=dev) for h in h_in]
    d_cols = [d_in[k] for k in idx]
    d_x = torch.empty(out_p, dtype=torch.int32, device=dev)
    d_z = torch.empty(out_p, dtype=torch.int32, device=dev)
    h2d = sum(h.numel() * 4 for h in h_in)
    d2h = 2 * out_p * 4

    side = torch.cuda.Stream(dev) if pin else None
    joined, copied = torch.cuda.Event(), torch.cuda.Event()

    def one(ev=None, overlap=True):
        if ev:
            ev[0].record()
        for d, h in zip(d_in, h_in):
            d.copy_(h, non_blocking=pin)
        if ev:
            ev[1].record()
        x, z = join_call(d_cols, d_x, d_z)
        if ev:
            ev[2].record()
        if overlap and side is not None:
            # the two output columns leave side by side: x on this stream, z
            # on a second one that waits for the join and is waited for
            joined.record()
            side.wait_event(joined)
            with torch.cuda.stream(side):
                h_z.copy_(z, non_blocking=True)
                copied.record(side)
            h_x.copy_(x, non_blocking=True)
            torch.cuda.current_stream().wait_event(copied)
        else:
            h_x.copy_(x, non_blocking=pin)
            if ev:
                ev[3].record()
            h_z.copy_(z, non_blocking=pin)
        if ev:
            ev[4].record()

    one()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        one()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    # two more steps with events between the parts: the columns copied side by
    # side as timed, then one after the other for each column's own rate
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    one(ev)
    torch.cuda.synchronize()
    both = ev[2].elapsed_time(ev[4])
    part = [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
    one(ev, overlap=False)
    torch.cuda.synchronize()
    part += [ev[2].elapsed_time(ev[3]), ev[3].elapsed_time(ev[4])]
    parts = {"h2d_ms": part[0], "join_ms": part[1], "d2h_both_ms": both,
             "d2h_both_gbs": 2 * out_p * 4 / max(both, 1e-6) / 1e6,
             "d2h_x_ms": part[2], "d2h_z_ms": part[3],
             "h2d_gbs": h2d / max(part[0], 1e-6) / 1e6, "d2h_x_gbs": out_p * 4 / max(part[2], 1e-6) / 1e6,
             "d2h_z_gbs": out_p * 4 / max(part[3], 1e-6) / 1e6}
    del d_in, d_x, d_z
    for rel in releases:
        rel()
    return {"value": out_p * steps / sum(times), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "host_memory": ("pinned, huge pages" if len(releases) == 2 else "pinned") if pin else "pageable",
            "ms_per_step": 1e3 * sum(times) / steps, "step_ms": [round(1e3 * t, 2) for t in times],
            "parts": parts, "gpu_numa": gpu,
            "out_columns": placement}


if __name__ == "__main__":
    main()
