"""Served execution: queries arriving over time are batched on the fly by
worker streams, and every result equals the query's result alone."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from paper_2206_04995_gb300.serve import Limits, Query, Server, summarize
from tests.gpu_util import host, inst_dev

pytestmark = pytest.mark.gpu


def stream(n, seed, rate):
    rng = np.random.default_rng(seed)
    arr = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        t = int(np.exp(rng.uniform(np.log(500), np.log(20_000))))
        inst = gen.two_table(np.random.default_rng(seed * 1000 + i), t, t, max(2, t // 10), max(2, int(t / 12.5)),
                             max(2, t // 20), 1.0)
        out.append(Query(i, "project" if rng.random() < 0.5 else "count", inst.r_key, inst.r_val, inst.s_key,
                         inst.s_val, float(arr[i])))
    return out


def alone(ctx, q):
    cols = inst_dev(gen.Instance("q", q.r_key, q.r_val, q.s_key, q.s_val))
    return ctx.join_count(*cols) if q.kind == "count" else ctx.join_project(*cols)


# realtime: arrivals 0.2 ms apart on average, well under one query's service time, so queues form
@pytest.mark.parametrize("realtime,rate", [(False, 0), (True, 5000.0)])
def test_served_equals_alone(realtime, rate):
    qs = stream(40, 3, rate or 1.0)
    srv = Server(0, workers=2, limits=Limits(max_batch=8, reserve_bytes=1 << 30))
    t0 = torch.cuda.Event(enable_timing=True)
    res = srv.run(qs, realtime=realtime)
    srv.close()
    assert [r.qid for r in res] == list(range(len(qs)))
    ctx = dim3.Context(0)
    for q, r in zip(qs, res):
        ref = alone(ctx, q)
        assert torch.equal(r.out_x, ref[0]) and torch.equal(r.out_z, ref[1]), f"query {q.qid}"
        if q.kind == "count":
            assert torch.equal(r.out_c, ref[2])
    ctx.close()
    assert max(r.batch_size for r in res) > 1, "no query was batched with another"
    s = summarize(res, max(r.done for r in res))
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["pairs"] == sum(r.pairs for r in res)
    del t0


def test_served_small_against_oracle():
    qs = stream(6, 11, 1.0)
    srv = Server(0, workers=2, limits=Limits(max_batch=4, reserve_bytes=1 << 30))
    res = srv.run(qs, realtime=False)
    srv.close()
    for q, r in zip(qs, res):
        if q.kind == "count":
            ox, oz, oc, _ = oracle.join_count(q.r_key, q.r_val, q.s_key, q.s_val)
            assert np.array_equal(host(r.out_c), oc.astype(np.int32))
        else:
            ox, oz, _ = oracle.join_project(q.r_key, q.r_val, q.s_key, q.s_val)
        assert np.array_equal(host(r.out_x), ox) and np.array_equal(host(r.out_z), oz)


@pytest.mark.parametrize("workers", [1, 3])
def test_chunked_output_and_big_queries(workers):
    """Results cut into many x-range chunks (a small chunk bound), big queries
    alone and small ones batched, equal the query's result alone; without
    keep, the parts handed to the consumer concatenate to the same result."""
    qs = stream(24, 5, 1.0)
    lim = Limits(max_batch=6, reserve_bytes=1 << 30, big_tuples=12_000, chunk_pairs=20_000)
    srv = Server(0, workers=workers, limits=lim)
    res = srv.run(qs, realtime=False)
    srv.close()
    assert max(r.chunks for r in res) > 3 and max(r.batch_size for r in res) > 1
    assert all(r.batch_size == 1 for q, r in zip(qs, res) if q.tuples > 12_000)
    got = {}

    def on_part(q, x, z, c):
        got.setdefault(q.qid, []).append((x.clone(), z.clone(), None if c is None else c.clone()))

    srv = Server(0, workers=workers, limits=lim, keep=False, on_part=on_part)
    res2 = srv.run(qs, realtime=False)
    srv.close()
    ctx = dim3.Context(0)
    for q, r, r2 in zip(qs, res, res2):
        ref = alone(ctx, q)
        assert torch.equal(r.out_x, ref[0]) and torch.equal(r.out_z, ref[1]), f"query {q.qid}"
        if q.kind == "count":
            assert torch.equal(r.out_c, ref[2])
        assert r2.pairs == ref[0].numel() and not r2.parts
        parts = got.get(q.qid, [])
        if parts:
            assert torch.equal(torch.cat([p[0] for p in parts]), ref[0])
            assert torch.equal(torch.cat([p[1] for p in parts]), ref[1])
            if q.kind == "count":
                assert torch.equal(torch.cat([p[2] for p in parts]), ref[2])
        else:
            assert ref[0].numel() == 0
    ctx.close()
