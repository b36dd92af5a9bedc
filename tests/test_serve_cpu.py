"""Host-side scheduling of the serving loop (no GPU): batch formation,
admission by free HBM, output chunking by the join-tuple bound, latency
statistics."""

from collections import deque

import numpy as np
import pytest

from paper_2206_04995_gb300.serve import (Limits, Query, admit, chunk_ranges, form_batch, percentile, plan_bytes,
                                          summarize)


def q(qid, kind="project", tuples=100):
    z = np.zeros(tuples // 2, np.int32)
    return Query(qid, kind, z, z, z, z, arrival=float(qid))


GB = 1 << 30


def test_fifo_same_kind_batches():
    queue = deque([q(0), q(1, "count"), q(2), q(3), q(4, "count")])
    b = form_batch(queue, Limits(max_batch=10, reserve_bytes=0), 100 * GB)
    assert [x.qid for x in b] == [0, 2, 3]
    assert [x.qid for x in queue] == [1, 4]  # order of the rest is kept
    b = form_batch(queue, Limits(max_batch=10, reserve_bytes=0), 100 * GB)
    assert [x.qid for x in b] == [1, 4] and not queue


def test_batch_size_and_tuple_limits():
    queue = deque(q(i, tuples=1000) for i in range(10))
    b = form_batch(queue, Limits(max_batch=4, max_tuples=10**9, reserve_bytes=0), 100 * GB)
    assert [x.qid for x in b] == [0, 1, 2, 3]
    b = form_batch(queue, Limits(max_batch=100, max_tuples=2500, reserve_bytes=0), 100 * GB)
    assert [x.qid for x in b] == [4, 5]


def test_memory_admission():
    big = q(0, tuples=10_000)
    queue = deque([big, q(1, tuples=10_000)])
    need = plan_bytes(big)
    # nothing fits: the head waits
    assert form_batch(queue, Limits(reserve_bytes=0), need - 1) == [] and len(queue) == 2
    # exactly the head fits
    b = form_batch(queue, Limits(reserve_bytes=0), need)
    assert [x.qid for x in b] == [0] and [x.qid for x in queue] == [1]
    # reserve is honoured
    assert form_batch(queue, Limits(reserve_bytes=GB), need + GB - 1) == []


def test_head_alone_even_over_tuple_budget():
    queue = deque([q(0, tuples=10**6), q(1, tuples=10)])
    b = form_batch(queue, Limits(max_tuples=100, reserve_bytes=0), 100 * GB)
    assert [x.qid for x in b] == [0]


def test_admit_output_bytes():
    assert admit(10 * GB, 2 * GB, (9 * GB) // 8, "project")
    assert not admit(10 * GB, 2 * GB, (9 * GB) // 8 + 1, "project")
    assert not admit(10 * GB, 2 * GB, (9 * GB) // 8, "count")


def test_percentiles_and_summary():
    assert percentile([], 50) != percentile([], 50)  # nan
    assert percentile([1, 2, 3, 4], 50) == pytest.approx(2.5)

    class R:
        def __init__(self, lat, pairs, bs):
            self.latency, self.pairs, self.batch_size, self.chunks = lat, pairs, bs, 1

    s = summarize([R(0.001, 10, 1), R(0.003, 30, 2)], 2.0)
    assert s["pairs"] == 40 and s["pairs_per_s"] == 20.0 and s["mean_batch"] == 1.5


def test_big_queries_run_alone():
    lim = Limits(max_batch=10, reserve_bytes=0, big_tuples=1000)
    queue = deque([q(0, tuples=500), q(1, tuples=5000), q(2, tuples=600), q(3, tuples=800)])
    b = form_batch(queue, lim, 100 * GB)
    assert [x.qid for x in b] == [0, 2, 3] and [x.qid for x in queue] == [1]
    b = form_batch(queue, lim, 100 * GB)
    assert [x.qid for x in b] == [1] and not queue


def test_chunk_ranges_cover_and_bound():
    rng = np.random.default_rng(0)
    outj = rng.integers(0, 1000, 500)
    outj[17] = 50_000  # one x above the chunk limit: a range of its own
    cum = np.concatenate([[0], np.cumsum(outj)])
    for lo, hi, lim in ((0, 500, 4000), (37, 411, 2500), (0, 500, 10**9), (5, 6, 10)):
        ch = chunk_ranges(cum, lo, hi, lim, n_z=800)
        assert ch[0][0] == lo and ch[-1][1] == hi
        assert all(a < b for a, b, _ in ch) and all(ch[i][1] == ch[i + 1][0] for i in range(len(ch) - 1))
        for a, b, bound in ch:
            oj = cum[b] - cum[a]
            assert bound == min(oj, (b - a) * 800)
            assert oj <= lim or b == a + 1
    assert chunk_ranges(cum, 3, 3, 100, 10) == []
