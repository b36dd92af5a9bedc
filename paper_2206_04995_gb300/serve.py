"""Continuous-batching server for Join-Project / Join-Count queries.

Queries arrive over time (e.g. a Poisson stream). Worker threads, each with
its own library context and CUDA stream, repeatedly take the waiting queries
that fit and run them while the other workers run theirs, so the work of
several batches overlaps on the device:

* a query of more than ``Limits.big_tuples`` input tuples runs alone, as a
  single-instance plan (the fastest kernels for large results);
* smaller queries of one kind (project or count) are batched -- up to
  ``max_batch`` queries and ``max_tuples`` tuples -- into ONE batched pass of
  the path (``dim3_batch_partition`` + one join over the batch plan, which
  keeps instances apart);
* the output is produced in x ranges: the plan's exact per-x join-tuple
  counts (|OUT_J| of each x, an upper bound of its pairs) cut the x ids into
  chunks of at most ``chunk_pairs`` bound, and each chunk waits for free HBM
  (admission), runs as one call into buffers of its bound's size, is handed
  to the consumer and released. A result larger than the free HBM is thus
  never held whole.

Every result is exactly the query's own Join-Project (or Join-Count). With
``keep`` the parts stay on the device in the ``Result`` (the caller releases
them); without it each part goes to ``on_part`` (if given) and is dropped,
and the Result keeps only the pair count.

The scheduling decisions (``form_batch``, ``admit``, ``chunk_ranges``) are
plain host logic without CUDA, so they are unit-tested on the CPU.
"""

from __future__ import annotations

import dataclasses
import threading
import time
from collections import deque

import numpy as np

# bytes of device memory per input tuple a planned batch holds besides its
# output: the tagged concatenation, ids, sort buffers and CSR (measured upper
# bound with margin)
PLAN_BYTES_PER_TUPLE = 96


@dataclasses.dataclass
class Query:
    qid: int
    kind: str                 # "project" or "count"
    r_key: object             # int32 columns: numpy arrays, CPU tensors (pinned is best) or device tensors
    r_val: object
    s_key: object
    s_val: object
    arrival: float = 0.0      # seconds after the stream start

    @property
    def tuples(self) -> int:
        return int(len(self.r_key) + len(self.s_key))


@dataclasses.dataclass
class Result:
    qid: int
    kind: str
    parts: list               # [(x, z, c or None)] device tensors in canonical order (keep), else []
    pairs: int
    arrival: float
    start: float
    done: float
    batch_size: int
    chunks: int = 1

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    def _cat(self, i):
        import torch

        if i == 2 and self.kind != "count":
            return None
        ts = [p[i] for p in self.parts]
        if not ts:
            return torch.empty(0, dtype=torch.int32, device="cuda")
        return ts[0] if len(ts) == 1 else torch.cat(ts)

    @property
    def out_x(self):
        return self._cat(0)

    @property
    def out_z(self):
        return self._cat(1)

    @property
    def out_c(self):
        return self._cat(2)


@dataclasses.dataclass
class Limits:
    max_batch: int = 64                 # queries per batch
    max_tuples: int = 8_000_000         # input tuples per batch
    reserve_bytes: int = 8 << 30        # HBM kept free for plans and other work
    big_tuples: int = 400_000           # queries with more input tuples run alone
    chunk_pairs: int = 1_500_000_000    # output bound (|OUT_J|) per emitting call


def plan_bytes(q: Query) -> int:
    return q.tuples * (PLAN_BYTES_PER_TUPLE + 8)


def form_batch(queue: deque, limits: Limits, free_bytes: int) -> list:
    """Take the next batch from the queue (FIFO): the oldest query alone if it
    is big, else the oldest query's kind and then later small queries of the
    same kind while the batch stays within max_batch, max_tuples and the free
    HBM minus the reserve. If even the oldest query's plan does not fit,
    nothing is taken (the caller waits for memory)."""
    if not queue:
        return []
    head = queue[0]
    budget = free_bytes - limits.reserve_bytes
    if plan_bytes(head) > budget:
        return []
    if head.tuples > limits.big_tuples:
        return [queue.popleft()]
    batch, tuples, need = [], 0, 0
    kept = deque()
    while queue:
        q = queue.popleft()
        fits = (q.kind == head.kind and q.tuples <= limits.big_tuples and len(batch) < limits.max_batch and
                (not batch or (tuples + q.tuples <= limits.max_tuples and need + plan_bytes(q) <= budget)))
        if fits:
            batch.append(q)
            tuples += q.tuples
            need += plan_bytes(q)
        else:
            kept.append(q)
    queue.extend(kept)
    return batch


def out_bytes(pairs: int, kind: str) -> int:
    return int(pairs) * (12 if kind == "count" else 8)


def admit(free_bytes: int, reserve: int, out_pairs: int, kind: str) -> bool:
    """Whether an output of out_pairs pairs (8 or 12 bytes each) fits the free
    HBM with half the reserve kept."""
    return out_bytes(out_pairs, kind) <= free_bytes - reserve // 2


def chunk_ranges(cum_outj: np.ndarray, x_begin: int, x_end: int, chunk_pairs: int, n_z: int) -> list:
    """Cut the x ids [x_begin, x_end) into consecutive ranges whose join-tuple
    total (an upper bound of their pairs) stays within chunk_pairs, a single x
    with more being a range of its own. cum_outj[i] = join tuples of the x
    ids < i (length n_x + 1). Returns [(a, b, bound)], bound = min(join
    tuples, (b - a) * n_z), the pairs the range can hold at most."""
    out = []
    a = x_begin
    while a < x_end:
        lim = cum_outj[a] + chunk_pairs
        b = int(np.searchsorted(cum_outj, lim, side="right")) - 1
        b = min(max(b, a + 1), x_end)
        bound = int(min(cum_outj[b] - cum_outj[a], (b - a) * n_z))
        out.append((a, b, bound))
        a = b
    return out


def percentile(values, p: float) -> float:
    if not values:
        return float("nan")
    return float(np.percentile(np.asarray(values, np.float64), p))


class Server:
    """Runs a stream of queries with `workers` threads (one CUDA stream and
    one library context each)."""

    def __init__(self, device: int = 0, workers: int = 2, limits: Limits | None = None, keep: bool = True,
                 on_part=None):
        import torch

        from . import dim3

        self.torch = torch
        self.dim3 = dim3
        self.device = torch.device("cuda", device)
        self.limits = limits or Limits()
        self.keep = keep
        self.on_part = on_part
        self.ctxs = [dim3.Context(device) for _ in range(workers)]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(workers)]
        self.queue: deque = deque()
        self.cv = threading.Condition()
        self.mem_lock = threading.Lock()
        self.results: list[Result] = []
        self.closed = False
        self.t0 = 0.0
        self.errors: list[BaseException] = []

    def close(self):
        for c in self.ctxs:
            c.close()

    # ------------------------------------------------------------ workers
    def _free_bytes(self) -> int:
        """Free HBM including what torch's caching allocator holds unused."""
        torch = self.torch
        free, _ = torch.cuda.mem_get_info(self.device)
        return int(free) + int(torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device))

    def _device_cols(self, q: Query):
        torch = self.torch
        out = []
        for a in (q.r_key, q.r_val, q.s_key, q.s_val):
            if isinstance(a, np.ndarray):
                a = torch.from_numpy(np.ascontiguousarray(a, np.int32))
            out.append(a.to(self.device, non_blocking=True))
        return out

    def _alloc_outputs(self, bound: int, kind: str):
        """Device buffers for `bound` pairs, once they fit the free HBM."""
        torch = self.torch
        n = max(int(bound), 1)
        for _ in range(120_000):  # wait up to ~10 minutes for other workers to release output
            with self.mem_lock:
                if admit(self._free_bytes(), self.limits.reserve_bytes, n, kind):
                    x = torch.empty(n, dtype=torch.int32, device=self.device)
                    z = torch.empty(n, dtype=torch.int32, device=self.device)
                    c = torch.empty(n, dtype=torch.int32, device=self.device) if kind == "count" else None
                    return x, z, c
            time.sleep(0.005)
        raise MemoryError(f"no room for an output of {n} pairs")

    def _run_batch(self, w: int, batch: list):
        torch = self.torch
        ctx, stream = self.ctxs[w], self.streams[w]
        start = time.perf_counter() - self.t0
        kind = batch[0].kind
        parts = [[] for _ in batch]
        pairs = [0] * len(batch)
        chunks = 0
        with torch.cuda.stream(stream):
            cols = [self._device_cols(q) for q in batch]
            plan = ctx.partition(*cols[0], stream=stream) if len(batch) == 1 else ctx.batch_partition(cols, stream=stream)
            try:
                info = plan.info
                lo = [0, info["n_x"]] if len(batch) == 1 else plan.instance_ranges()
                outj = plan.export("outj_x", stream=stream)
                cum = torch.cat([torch.zeros(1, dtype=torch.int64, device=self.device), torch.cumsum(outj, 0)])
                cum = cum.cpu().numpy()
                for a, b, bound in chunk_ranges(cum, 0, info["n_x"], self.limits.chunk_pairs, info["n_z"]):
                    if bound == 0:
                        continue
                    bx, bz, bc = self._alloc_outputs(bound, kind)
                    if kind == "count":
                        x, z, c = plan.join_count(a, b, out_x=bx, out_z=bz, out_c=bc, stream=stream)
                    else:
                        x, z = plan.join_project(a, b, out_x=bx, out_z=bz, stream=stream)
                        c = None
                    chunks += 1
                    # split the chunk among the queries whose x ids it covers
                    if len(batch) == 1:
                        spans = [(0, 0, x.numel())]
                    else:
                        rc = plan.row_counts(a, b, stream=stream)
                        off = torch.cat([torch.zeros(1, dtype=torch.int64, device=self.device),
                                         torch.cumsum(rc, 0)]).cpu().numpy()
                        spans = []
                        for t in range(len(batch)):
                            ta, tb = max(lo[t], a), min(lo[t + 1], b)
                            if tb > ta:
                                spans.append((t, int(off[ta - a]), int(off[tb - a])))
                    for t, p0, p1 in spans:
                        if p1 <= p0:
                            continue
                        px, pz, pc = x[p0:p1], z[p0:p1], (c[p0:p1] if c is not None else None)
                        pairs[t] += p1 - p0
                        if self.on_part is not None:
                            self.on_part(batch[t], px, pz, pc)
                        if self.keep:
                            parts[t].append((px, pz, pc))
                    del x, z, c, bx, bz, bc
            finally:
                plan.close()
            stream.synchronize()
        done = time.perf_counter() - self.t0
        return [Result(q.qid, q.kind, parts[t], pairs[t], q.arrival, start, done, len(batch), chunks)
                for t, q in enumerate(batch)]

    def _worker(self, w: int):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.cv:
                while True:
                    if self.queue:
                        batch = form_batch(self.queue, self.limits, self._free_bytes())
                        if batch:
                            break
                    elif self.closed:
                        return
                    self.cv.wait(timeout=0.01)
            try:
                res = self._run_batch(w, batch)
            except BaseException as e:  # noqa: BLE001
                self.errors.append(e)
                with self.cv:
                    self.closed = True
                    self.queue.clear()
                    self.cv.notify_all()
                return
            with self.cv:
                self.results.extend(res)
                self.cv.notify_all()

    # -------------------------------------------------------------- stream
    def run(self, queries: list, realtime: bool = True) -> list:
        """Feed `queries` at their arrival times (or all at once when
        realtime is False) and return every Result once all are served."""
        self.results = []
        self.closed = False
        self.errors = []
        self.t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(w,), daemon=True) for w in range(len(self.ctxs))]
        for t in threads:
            t.start()
        for q in sorted(queries, key=lambda q: q.arrival):
            if realtime:
                delay = q.arrival - (time.perf_counter() - self.t0)
                if delay > 0:
                    time.sleep(delay)
            else:
                q.arrival = time.perf_counter() - self.t0
            with self.cv:
                if self.closed:
                    break
                self.queue.append(q)
                self.cv.notify_all()
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for t in threads:
            t.join()
        if self.errors:
            raise self.errors[0]
        return sorted(self.results, key=lambda r: r.qid)


def summarize(results: list, wall_s: float) -> dict:
    lat = [r.latency for r in results]
    pairs = sum(r.pairs for r in results)
    return {"queries": len(results), "pairs": pairs, "wall_s": wall_s, "pairs_per_s": pairs / wall_s,
            "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "mean_batch": float(np.mean([r.batch_size for r in results])) if results else 0.0,
            "chunks": int(sum(r.chunks for r in results if r.batch_size == 1))}
