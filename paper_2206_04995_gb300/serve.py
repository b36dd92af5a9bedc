"""Continuous-batching server for Join-Project / Join-Count queries.

Queries arrive over time (e.g. a Poisson stream). Worker threads, each with
its own CUDA stream, repeatedly take the waiting queries that fit -- same
kind (project or count), up to a batch size and tuple budget, and only as
many as the free HBM admits -- and run them as ONE batched pass of the path
(``dim3_batch_partition`` + one join over the batch plan). Queries that
arrive while batches are on the GPU wait in the queue and join the next
batch a worker forms, so work of several batches overlaps on the device.
Every result is exactly the query's own Join-Project (the batch keeps
instances apart), returned as device tensors the caller releases after use.

The scheduling decisions (``form_batch``, ``admit``) are plain host logic
without CUDA, so they are unit-tested on the CPU.
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
    r_key: np.ndarray
    r_val: np.ndarray
    s_key: np.ndarray
    s_val: np.ndarray
    arrival: float = 0.0      # seconds after the stream start

    @property
    def tuples(self) -> int:
        return int(self.r_key.size + self.s_key.size)


@dataclasses.dataclass
class Result:
    qid: int
    kind: str
    out_x: object             # device tensors (torch), released by the caller
    out_z: object
    out_c: object | None
    arrival: float
    start: float
    done: float
    batch_size: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def pairs(self) -> int:
        return int(self.out_x.numel())


@dataclasses.dataclass
class Limits:
    max_batch: int = 64                 # queries per batch
    max_tuples: int = 8_000_000         # input tuples per batch
    reserve_bytes: int = 8 << 30        # HBM kept free for outputs and other work


def plan_bytes(q: Query) -> int:
    return q.tuples * (PLAN_BYTES_PER_TUPLE + 8)


def form_batch(queue: deque, limits: Limits, free_bytes: int) -> list:
    """Take the next batch from the queue (FIFO): the oldest query's kind,
    then later queries of the same kind while the batch stays within
    max_batch, max_tuples and the free HBM minus the reserve. The oldest query
    is taken alone if nothing else fits; if even it does not fit, nothing is
    taken (the caller waits for memory)."""
    if not queue:
        return []
    head = queue[0]
    budget = free_bytes - limits.reserve_bytes
    if plan_bytes(head) > budget:
        return []
    batch, tuples, need = [], 0, 0
    kept = deque()
    while queue:
        q = queue.popleft()
        fits = (q.kind == head.kind and len(batch) < limits.max_batch and
                (not batch or (tuples + q.tuples <= limits.max_tuples and need + plan_bytes(q) <= budget)))
        if fits:
            batch.append(q)
            tuples += q.tuples
            need += plan_bytes(q)
        else:
            kept.append(q)
    queue.extend(kept)
    return batch


def admit(free_bytes: int, reserve: int, out_pairs: int, kind: str) -> bool:
    """Whether a batch's output (8 or 12 bytes per pair) fits the free HBM."""
    return out_pairs * (12 if kind == "count" else 8) <= free_bytes - reserve // 2


def percentile(values, p: float) -> float:
    if not values:
        return float("nan")
    return float(np.percentile(np.asarray(values, np.float64), p))


class Server:
    """Runs a stream of queries with `workers` threads (one CUDA stream each)."""

    def __init__(self, device: int = 0, workers: int = 2, limits: Limits | None = None):
        import torch

        from . import dim3

        self.torch = torch
        self.device = torch.device("cuda", device)
        self.limits = limits or Limits()
        self.ctxs = [dim3.Context(device) for _ in range(workers)]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(workers)]
        self.queue: deque = deque()
        self.cv = threading.Condition()
        self.results: list[Result] = []
        self.closed = False
        self.t0 = 0.0
        self.errors: list[BaseException] = []

    def close(self):
        for c in self.ctxs:
            c.close()

    # ------------------------------------------------------------ workers
    def _free_bytes(self) -> int:
        free, _ = self.torch.cuda.mem_get_info(self.device)
        return int(free)

    def _run_batch(self, w: int, batch: list):
        torch = self.torch
        ctx, stream = self.ctxs[w], self.streams[w]
        start = time.perf_counter() - self.t0
        with torch.cuda.stream(stream):
            cols = []
            for q in batch:
                cols.append([torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory().to(
                    self.device, non_blocking=True) for a in (q.r_key, q.r_val, q.s_key, q.s_val)])
            plan = ctx.batch_partition(cols, stream=stream)
            try:
                rc = plan.row_counts(stream=stream)
                lo = plan.instance_ranges()
                cs = torch.cumsum(torch.cat([torch.zeros(1, dtype=torch.int64, device=self.device), rc]), 0)
                bounds = cs[torch.tensor(lo, device=self.device)].tolist()
                total = bounds[-1]
                kind = batch[0].kind
                # wait until the output fits (other workers release theirs)
                for _ in range(6000):
                    if admit(self._free_bytes(), self.limits.reserve_bytes, total, kind):
                        break
                    time.sleep(0.005)
                if kind == "count":
                    x, z, c = plan.join_count(stream=stream)
                else:
                    x, z = plan.join_project(stream=stream)
                    c = None
            finally:
                plan.close()
            stream.synchronize()
        done = time.perf_counter() - self.t0
        out = []
        for t, q in enumerate(batch):
            a, b = bounds[t], bounds[t + 1]
            out.append(Result(q.qid, q.kind, x[a:b], z[a:b], None if c is None else c[a:b], q.arrival, start,
                              done, len(batch)))
        return out

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
            "mean_batch": float(np.mean([r.batch_size for r in results])) if results else 0.0}
