"""Thin Python binding of the C ABI in ``include/dim3.h`` (ctypes).

Argument marshalling only: torch supplies device memory and streams; every
step of the Join-Project path runs in the CUDA kernels of ``libdim3.so``.
There is no CPU fallback: without the library (or a GB300) calls raise.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

DIM3_OK = 0
DIM3_ERR_ARG = -1
DIM3_ERR_CUDA = -2
DIM3_ERR_NOMEM = -3
DIM3_ERR_CAPACITY = -4
DIM3_ERR_TIMEOUT = -5
DIM3_ERR_OVERFLOW = -6
DIM3_ERR_UNSUPPORTED = -7

DENSE_AUTO, DENSE_TC, DENSE_POPC, DENSE_PROBE = 0, 1, 2, 3
OPT_THETA_Z, OPT_DENSE_VARIANT, OPT_BITMAP_ROW_MIN, OPT_LIGHT_ROW_MAX, OPT_TIMING = 1, 2, 3, 4, 5
OPT_EMIT_ROWS = 6
AGG_COUNT, AGG_SUM, AGG_MIN, AGG_MAX, AGG_AVG = 0, 1, 2, 3, 4
FN_MUL, FN_ADD, FN_LEFT, FN_RIGHT = 0, 1, 2, 3
OPT_TWO_PASS = 7
OPT_ID_CHUNK_MAX = 8
OPT_PATH = 9
OPT_TILE_WORDS = 10
OPT_DENSE_TILE_N = 11
OPT_EMIT_PIPELINE = 12
PATH_AUTO, PATH_HYBRID, PATH_CLASSICAL = 0, 1, 2
PHASES = {"map": 0, "partition": 1, "dense_ec": 2, "sparse_count": 3, "sparse_emit": 4, "dense_tc": 5}

TABLES = {
    "dict_x": (1, torch.int32), "dict_y": (2, torch.int32), "dict_z": (3, torch.int32),
    "r_rowptr": (4, torch.int64), "r_col": (5, torch.int32), "m_z": (6, torch.int32),
    "dense_z": (7, torch.uint8), "ss_rowptr": (8, torch.int64), "ss_col": (9, torch.int32),
    "deg_s": (10, torch.int32), "outj_x": (11, torch.int64),
}


class Dim3Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dim3 error {status}: {msg}")
        self.status = status


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_r", "n_s", "n_r_kept", "n_s_distinct", "n_x", "n_y", "n_z", "n_z_dense", "n_y_dense",
        "n_s_sparse", "n_y_bitmap", "out_j", "n_z_cached")] + [("theta_z", ctypes.c_int32),
                                                               ("dense_variant", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class EdgeTable(ctypes.Structure):
    """dim3_edge_table: one relation R_i(x_i, x_{i+1}) of a multi-way join."""
    _fields_ = [("d_a", ctypes.c_void_p), ("d_b", ctypes.c_void_p), ("n", ctypes.c_int64)]


class CacheInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_entries", "n_list", "space", "n_x")]


class Instance(ctypes.Structure):
    """dim3_instance: one instance of a batch (device column pointers)."""
    _fields_ = [("r_key", ctypes.c_void_p), ("r_val", ctypes.c_void_p), ("nr", ctypes.c_int64),
                ("s_key", ctypes.c_void_p), ("s_val", ctypes.c_void_p), ("ns", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdim3.so (building it in-tree first if it is missing or stale
    and nvcc is available). Raises if the library cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            try:
                _build.build()
            except Exception as e:  # noqa: BLE001
                if not os.path.exists(_build.LIB):
                    raise RuntimeError(f"libdim3.so is missing and could not be built: {e}") from e
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libdim3.so is missing; run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        P, I64, I32, INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        sig = {
            "dim3_version": ([], INT),
            "dim3_last_error": ([], ctypes.c_char_p),
            "dim3_ctx_create": ([ctypes.POINTER(P), INT], INT),
            "dim3_ctx_destroy": ([P], INT),
            "dim3_ctx_set_option": ([P, INT, I64], INT),
            "dim3_ctx_timing": ([P, INT, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I64), INT], INT),
            "dim3_launch_count": ([ctypes.POINTER(I64)], INT),
            "dim3_map": ([P, P, I64, P, P, ctypes.POINTER(I64), P], INT),
            "dim3_partition": ([P, P, P, I64, P, P, I64, I32, ctypes.POINTER(P), ctypes.POINTER(PlanInfo), P], INT),
            "dim3_partition_ids": ([P, P, P, I64, P, P, I64, I64, I64, I64, I32, ctypes.POINTER(P),
                                    ctypes.POINTER(PlanInfo), P], INT),
            "dim3_map_tuples": ([P, P, ctypes.c_int, ctypes.c_uint32, I64, P, P, ctypes.POINTER(I64), P], INT),
            "dim3_gather_i32": ([P, P, I64, P, I64, P, P], INT),
            "dim3_selftest_wait_timeout": ([P, ctypes.c_double, P], INT),
            "dim3_ctx_set_f1_costs": ([P, ctypes.c_double, ctypes.c_double, ctypes.c_double], INT),
            "dim3_ctx_last_path": ([P], INT),
            "dim3_join_aggregate": ([P, P, P, P, I64, P, P, P, I64, ctypes.c_int, ctypes.c_int, P, P, P, I64,
                                     ctypes.POINTER(I64), P], INT),
            "dim3_groupby_aggregate": ([P, P, P, I64, P, P, I64, ctypes.c_int, P, P, I64, ctypes.POINTER(I64), P],
                                       INT),
            "dim3_mjp_sizes": ([P, ctypes.c_int, P, P, P, P], INT),
            "dim3_mjp_plan": ([ctypes.c_int, P, P, P, P, P, P], INT),
            "dim3_mjp_execute": ([P, ctypes.c_int, P, P, P, P, I64, ctypes.POINTER(I64), P], INT),
            "dim3_cache_build": ([P, P, P, I64, P, P, I64, I32, I64, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(P), ctypes.POINTER(CacheInfo), P], INT),
            "dim3_cache_export": ([P, P, P, P, P, P, P, P], INT),
            "dim3_cache_destroy": ([P], INT),
            "dim3_partition_cached": ([P, P, P, I64, P, P, I64, P, I32, ctypes.POINTER(P), ctypes.POINTER(PlanInfo),
                                       P], INT),
            "dim3_plan_get_info": ([P, ctypes.POINTER(PlanInfo)], INT),
            "dim3_plan_row_counts": ([P, P, I64, I64, P, P], INT),
            "dim3_plan_join_project": ([P, P, I64, I64, P, P, I64, ctypes.POINTER(I64), P], INT),
            "dim3_plan_join_count": ([P, P, I64, I64, P, P, P, I64, ctypes.POINTER(I64), P], INT),
            "dim3_plan_export": ([P, INT, P, I64, P], INT),
            "dim3_plan_destroy": ([P], INT),
            "dim3_join_project": ([P, P, P, I64, P, P, I64, P, P, I64, ctypes.POINTER(I64), P], INT),
            "dim3_join_count": ([P, P, P, I64, P, P, I64, P, P, P, I64, ctypes.POINTER(I64), P], INT),
            "dim3_batch_partition": ([P, INT, P, I32, ctypes.POINTER(P), ctypes.POINTER(PlanInfo), P], INT),
            "dim3_plan_instance_ranges": ([P, P], INT),
            "dim3_batch_join_project": ([P, INT, P, P, P, I64, P, ctypes.POINTER(I64), P], INT),
            "dim3_batch_join_count": ([P, INT, P, P, P, P, I64, P, ctypes.POINTER(I64), P], INT),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return _lib


def launch_count() -> int:
    """Kernels launched by libdim3.so in this process."""
    n = ctypes.c_int64()
    _check(load().dim3_launch_count(ctypes.byref(n)))
    return n.value


def _check(rc: int):
    if rc != DIM3_OK:
        raise Dim3Error(rc, load().dim3_last_error().decode(errors="replace"))


def _ptr(t: torch.Tensor | None):
    return None if t is None or t.numel() == 0 else ctypes.c_void_p(t.data_ptr())


def _col(t: torch.Tensor, device: torch.device, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.int32 or t.device != device or t.dim() != 1 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous 1-D int32 tensor on {device}")
    return t


def _stream(device, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A library context on one CUDA device (``dim3_ctx``)."""

    def __init__(self, device: int = 0):
        self._lib = load()
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        _check(self._lib.dim3_ctx_create(ctypes.byref(h), device))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dim3_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def set_option(self, option: int, value: int):
        _check(self._lib.dim3_ctx_set_option(self._h, option, int(value)))

    def timing(self, reset: bool = False) -> dict:
        """{phase: (total_ms, intervals)} recorded while OPT_TIMING is on."""
        out = {}
        for name, ph in PHASES.items():
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            _check(self._lib.dim3_ctx_timing(self._h, ph, ctypes.byref(ms), ctypes.byref(n), 0))
            out[name] = (ms.value, n.value)
        if reset:
            _check(self._lib.dim3_ctx_timing(self._h, 0, None, None, 1))
        return out

    # -------------------------------------------------------------- mapping
    def map(self, vals: torch.Tensor, stream=None):
        """Order-preserving ids of a column: (ids, dict)."""
        vals = _col(vals, self.device, "vals")
        n = vals.numel()
        ids = torch.empty(n, dtype=torch.int32, device=self.device)
        d = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        nd = ctypes.c_int64()
        _check(self._lib.dim3_map(self._h, _ptr(vals), n, _ptr(ids), _ptr(d), ctypes.byref(nd),
                                  _stream(self.device, stream)))
        return ids, d[: nd.value]

    def map_tuples(self, cols, unsigned_mask: int = 0, stream=None):
        """Ranks of k-column tuples in lexicographic order: (ids, first), first[id]
        = smallest row with that tuple (``dim3_map_tuples``)."""
        cols = [_col(c, self.device, f"col{i}") for i, c in enumerate(cols)]
        n = cols[0].numel() if cols else 0
        if any(c.numel() != n for c in cols):
            raise ValueError("column lengths differ")
        ptrs = (ctypes.c_void_p * max(len(cols), 1))(*[_ptr(c) for c in cols])
        ids = torch.empty(n, dtype=torch.int32, device=self.device)
        first = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        nd = ctypes.c_int64()
        _check(self._lib.dim3_map_tuples(self._h, ptrs, len(cols), int(unsigned_mask) & 0xFFFFFFFF, n, _ptr(ids),
                                         _ptr(first), ctypes.byref(nd), _stream(self.device, stream)))
        return ids, first[: nd.value]

    def selftest_wait_timeout(self, seconds: float = 0.05, stream=None) -> int:
        """Run ``dim3_selftest_wait_timeout``; returns its status (DIM3_ERR_TIMEOUT
        when the bounded wait gave up as intended)."""
        return self._lib.dim3_selftest_wait_timeout(self._h, float(seconds), _stream(self.device, stream))

    def gather(self, src, idx, stream=None):
        """src[idx] through ``dim3_gather_i32`` (int32)."""
        src, idx = _col(src, self.device, "src"), _col(idx, self.device, "idx")
        out = torch.empty(idx.numel(), dtype=torch.int32, device=self.device)
        _check(self._lib.dim3_gather_i32(self._h, _ptr(src), src.numel(), _ptr(idx), idx.numel(), _ptr(out),
                                         _stream(self.device, stream)))
        return out

    # ------------------------------------------------------------ partition
    def partition_ids(self, r_y, r_x, s_y, s_z, n_x: int, n_y: int, n_z: int, theta_z: int = -1,
                      stream=None) -> "Plan":
        """Plan over pre-mapped ids (mapping skipped, ``dim3_partition_ids``)."""
        r_y, r_x = _col(r_y, self.device, "r_y"), _col(r_x, self.device, "r_x")
        s_y, s_z = _col(s_y, self.device, "s_y"), _col(s_z, self.device, "s_z")
        if r_y.numel() != r_x.numel() or s_y.numel() != s_z.numel():
            raise ValueError("column lengths differ")
        h = ctypes.c_void_p()
        info = PlanInfo()
        _check(self._lib.dim3_partition_ids(self._h, _ptr(r_y), _ptr(r_x), r_y.numel(), _ptr(s_y), _ptr(s_z),
                                            s_y.numel(), int(n_x), int(n_y), int(n_z), int(theta_z),
                                            ctypes.byref(h), ctypes.byref(info), _stream(self.device, stream)))
        return Plan(self, h, info, stream)

    def set_f1_costs(self, t_map: float, t_rand: float, t_hash: float):
        """Constants of f1 (Section 2.6), seconds."""
        _check(self._lib.dim3_ctx_set_f1_costs(self._h, float(t_map), float(t_rand), float(t_hash)))

    def last_path(self) -> int:
        """Path of the last one-call join: 1 hybrid, 2 classical."""
        return int(self._lib.dim3_ctx_last_path(self._h))

    # ------------------------------------------------------- Join-Aggregate
    def join_aggregate(self, r_key, r_val, r_v, s_key, s_val, s_u, agg: int, fn: int = FN_MUL, out=None,
                       stream=None):
        """G_{x,z} agg(f(R.v, S.u)) (``dim3_join_aggregate``): (x, z, value),
        value int64, or float64 for AVG. ``out`` = preallocated (x, z, value)
        makes it one C call; otherwise a sizing call comes first."""
        cols = [_col(t, self.device, n) for t, n in ((r_key, "r_key"), (r_val, "r_val"), (r_v, "r_v"),
                                                      (s_key, "s_key"), (s_val, "s_val"), (s_u, "s_u"))]
        if not (cols[0].numel() == cols[1].numel() == cols[2].numel()) or not (
                cols[3].numel() == cols[4].numel() == cols[5].numel()):
            raise ValueError("column lengths differ")
        st = _stream(self.device, stream)
        n = ctypes.c_int64()
        args = [self._h, _ptr(cols[0]), _ptr(cols[1]), _ptr(cols[2]), cols[0].numel(), _ptr(cols[3]), _ptr(cols[4]),
                _ptr(cols[5]), cols[3].numel(), int(agg), int(fn)]
        if out is not None:
            ox, oz, ov = out
            _check(self._lib.dim3_join_aggregate(*args, _ptr(ox), _ptr(oz), _ptr(ov), ox.numel(), ctypes.byref(n),
                                                 st))
            return ox[: n.value], oz[: n.value], ov[: n.value]
        rc = self._lib.dim3_join_aggregate(*args, None, None, None, 0, ctypes.byref(n), st)
        if rc not in (DIM3_OK, DIM3_ERR_CAPACITY):
            _check(rc)
        m = n.value
        x = torch.empty(m, dtype=torch.int32, device=self.device)
        z = torch.empty(m, dtype=torch.int32, device=self.device)
        v = torch.empty(m, dtype=torch.float64 if agg == AGG_AVG else torch.int64, device=self.device)
        if m:
            _check(self._lib.dim3_join_aggregate(*args, _ptr(x), _ptr(z), _ptr(v), m, ctypes.byref(n), st))
        return x, z, v

    def groupby_aggregate(self, r_key, r_val, s_key, s_val, agg: int, stream=None):
        """G_x agg(z) over R(x, y) join S(z, y) (``dim3_groupby_aggregate``): (x, value)."""
        cols = [_col(t, self.device, n) for t, n in ((r_key, "r_key"), (r_val, "r_val"), (s_key, "s_key"),
                                                      (s_val, "s_val"))]
        if cols[0].numel() != cols[1].numel() or cols[2].numel() != cols[3].numel():
            raise ValueError("column lengths differ")
        st = _stream(self.device, stream)
        n = ctypes.c_int64()
        args = [self._h, _ptr(cols[0]), _ptr(cols[1]), cols[0].numel(), _ptr(cols[2]), _ptr(cols[3]),
                cols[2].numel(), int(agg)]
        rc = self._lib.dim3_groupby_aggregate(*args, None, None, 0, ctypes.byref(n), st)
        if rc not in (DIM3_OK, DIM3_ERR_CAPACITY):
            _check(rc)
        m = n.value
        x = torch.empty(m, dtype=torch.int32, device=self.device)
        v = torch.empty(m, dtype=torch.float64 if agg == AGG_AVG else torch.int64, device=self.device)
        if m:
            _check(self._lib.dim3_groupby_aggregate(*args, _ptr(x), _ptr(v), m, ctypes.byref(n), st))
        return x, v

    # ------------------------------------------------------------------ MJP
    # Section 4.2 cost constants (seconds): bag join per input row and per
    # result pair, Join-Project per input row, per join tuple, per result pair
    MJP_COSTS = (3.0e-10, 4.0e-11, 4.0e-10, 1.0e-12, 1.5e-12)

    def _edges(self, tables):
        cols = []
        arr = (EdgeTable * len(tables))()
        for i, (a, b) in enumerate(tables):
            a, b = _col(a, self.device, f"R{i + 1}.a"), _col(b, self.device, f"R{i + 1}.b")
            if a.numel() != b.numel():
                raise ValueError(f"table {i + 1}: column lengths differ")
            cols.append((a, b))
            arr[i] = EdgeTable(a.data_ptr() if a.numel() else None, b.data_ptr() if b.numel() else None, a.numel())
        return arr, cols

    def mjp_sizes(self, tables, stream=None):
        """Exact |OUT_J_i| and |OUT_P_i| of the line query (``dim3_mjp_sizes``)."""
        arr, _keep = self._edges(tables)
        k = len(tables)
        oj, op = (ctypes.c_double * k)(), (ctypes.c_double * k)()
        _check(self._lib.dim3_mjp_sizes(self._h, k, arr, oj, op, _stream(self.device, stream)))
        return list(oj), list(op)

    @staticmethod
    def mjp_plan(r_size, out_j, out_p, costs=MJP_COSTS):
        """Deduplication placement of Section 4.2's DP (``dim3_mjp_plan``):
        (dedup flags, estimated cost)."""
        k = len(r_size)
        D = ctypes.c_double * k
        dedup = (ctypes.c_int * k)()
        cost = ctypes.c_double()
        _check(load().dim3_mjp_plan(k, D(*r_size), D(*out_j), D(*out_p), (ctypes.c_double * 5)(*costs), dedup,
                                    ctypes.byref(cost)))
        return [bool(v) for v in dedup], cost.value

    def mjp_execute(self, tables, dedup, out=None, stream=None):
        """Run a placement of the line query (``dim3_mjp_execute``): (x_1, x_{k+1})."""
        arr, _keep = self._edges(tables)
        k = len(tables)
        flags = (ctypes.c_int * k)(*[int(bool(v)) for v in dedup])
        st = _stream(self.device, stream)
        n = ctypes.c_int64()
        if out is None:
            rc = self._lib.dim3_mjp_execute(self._h, k, arr, flags, None, None, 0, ctypes.byref(n), st)
            if rc not in (DIM3_OK, DIM3_ERR_CAPACITY):
                _check(rc)
            out = (torch.empty(n.value, dtype=torch.int32, device=self.device),
                   torch.empty(n.value, dtype=torch.int32, device=self.device))
            if n.value == 0:
                return out
        x, z = out
        _check(self._lib.dim3_mjp_execute(self._h, k, arr, flags, _ptr(x), _ptr(z), min(x.numel(), z.numel()),
                                          ctypes.byref(n), st))
        return x[: n.value], z[: n.value]

    # Section 3 cost constants measured on GB300 (seconds): one SparseBMM join
    # tuple, one DenseEC (x, z) evaluation
    T_SPARSE = 1.2e-12
    T_DENSE = 1.1e-11

    def cache_build(self, r_key, r_val, s_key, s_val, budget: int, theta_z: int = -1, t_sparse: float = T_SPARSE,
                    t_dense: float = T_DENSE, stream=None) -> "ResultCache":
        """Partial result cache of the tables within ``budget`` entries
        (``dim3_cache_build``)."""
        r_key, r_val = _col(r_key, self.device, "r_key"), _col(r_val, self.device, "r_val")
        s_key, s_val = _col(s_key, self.device, "s_key"), _col(s_val, self.device, "s_val")
        if r_key.numel() != r_val.numel() or s_key.numel() != s_val.numel():
            raise ValueError("column lengths differ")
        h = ctypes.c_void_p()
        info = CacheInfo()
        _check(self._lib.dim3_cache_build(self._h, _ptr(r_key), _ptr(r_val), r_key.numel(), _ptr(s_key),
                                          _ptr(s_val), s_key.numel(), int(theta_z), int(budget), float(t_sparse),
                                          float(t_dense), ctypes.byref(h), ctypes.byref(info),
                                          _stream(self.device, stream)))
        return ResultCache(self, h, info)

    def partition_cached(self, r_key, r_val, s_key, s_val, cache: "ResultCache", theta_z: int = -1,
                         stream=None) -> "Plan":
        """Plan whose results include ``cache``'s pairs (``dim3_partition_cached``)."""
        r_key, r_val = _col(r_key, self.device, "r_key"), _col(r_val, self.device, "r_val")
        s_key, s_val = _col(s_key, self.device, "s_key"), _col(s_val, self.device, "s_val")
        if r_key.numel() != r_val.numel() or s_key.numel() != s_val.numel():
            raise ValueError("column lengths differ")
        h = ctypes.c_void_p()
        info = PlanInfo()
        _check(self._lib.dim3_partition_cached(self._h, _ptr(r_key), _ptr(r_val), r_key.numel(), _ptr(s_key),
                                               _ptr(s_val), s_key.numel(), cache._h, int(theta_z), ctypes.byref(h),
                                               ctypes.byref(info), _stream(self.device, stream)))
        return Plan(self, h, info, stream)

    def partition(self, r_key, r_val, s_key, s_val, theta_z: int = -1, stream=None) -> "Plan":
        r_key, r_val = _col(r_key, self.device, "r_key"), _col(r_val, self.device, "r_val")
        s_key, s_val = _col(s_key, self.device, "s_key"), _col(s_val, self.device, "s_val")
        if r_key.numel() != r_val.numel() or s_key.numel() != s_val.numel():
            raise ValueError("column lengths differ")
        h = ctypes.c_void_p()
        info = PlanInfo()
        _check(self._lib.dim3_partition(self._h, _ptr(r_key), _ptr(r_val), r_key.numel(), _ptr(s_key), _ptr(s_val),
                                        s_key.numel(), int(theta_z), ctypes.byref(h), ctypes.byref(info),
                                        _stream(self.device, stream)))
        return Plan(self, h, info, stream)

    # -------------------------------------------------------- one-call path
    def join_project(self, r_key, r_val, s_key, s_val, out_x=None, out_z=None, stream=None):
        """Pi_{x,z}(R join_y S): (out_x, out_z) in canonical order. With
        preallocated outputs the single C call ``dim3_join_project`` runs;
        otherwise a plan sizes the result first."""
        if out_x is not None:
            return self._join_call(False, r_key, r_val, s_key, s_val, out_x, out_z, None, stream)
        plan = self.partition(r_key, r_val, s_key, s_val, stream=stream)
        try:
            return plan.join_project(stream=stream)
        finally:
            plan.close()

    def join_count(self, r_key, r_val, s_key, s_val, out_x=None, out_z=None, out_c=None, stream=None):
        """Join-Aggregate COUNT: (out_x, out_z, out_cnt)."""
        if out_x is not None:
            return self._join_call(True, r_key, r_val, s_key, s_val, out_x, out_z, out_c, stream)
        plan = self.partition(r_key, r_val, s_key, s_val, stream=stream)
        try:
            return plan.join_count(stream=stream)
        finally:
            plan.close()

    # -------------------------------------------------------------- batches
    def _instances(self, instances):
        arr = (Instance * len(instances))()
        for i, (rk, rv, sk, sv) in enumerate(instances):
            rk, rv = _col(rk, self.device, "r_key"), _col(rv, self.device, "r_val")
            sk, sv = _col(sk, self.device, "s_key"), _col(sv, self.device, "s_val")
            if rk.numel() != rv.numel() or sk.numel() != sv.numel():
                raise ValueError(f"instance {i}: column lengths differ")
            arr[i] = Instance(rk.data_ptr() if rk.numel() else None, rv.data_ptr() if rv.numel() else None,
                              rk.numel(), sk.data_ptr() if sk.numel() else None,
                              sv.data_ptr() if sv.numel() else None, sk.numel())
        return arr

    def batch_partition(self, instances, theta_z: int = -1, stream=None) -> "Plan":
        """A plan over a batch of (r_key, r_val, s_key, s_val) instances."""
        arr = self._instances(instances)
        h = ctypes.c_void_p()
        info = PlanInfo()
        _check(self._lib.dim3_batch_partition(self._h, len(instances), arr, int(theta_z), ctypes.byref(h),
                                              ctypes.byref(info), _stream(self.device, stream)))
        return Plan(self, h, info, stream, n_inst=len(instances))

    def batch_join_project(self, instances, out_x=None, out_z=None, stream=None):
        """Eq. 1 for every instance of a batch in one pass: (out_x, out_z,
        per-instance pair counts); instance t's pairs follow instance t-1's."""
        return self._batch(False, instances, out_x, out_z, None, stream)

    def batch_join_count(self, instances, out_x=None, out_z=None, out_c=None, stream=None):
        return self._batch(True, instances, out_x, out_z, out_c, stream)

    def _batch(self, counts, instances, out_x, out_z, out_c, stream):
        if out_x is None:
            plan = self.batch_partition(instances, stream=stream)
            try:
                res = plan.join_count(stream=stream) if counts else plan.join_project(stream=stream)
                rc = plan.row_counts(stream=stream)
                lo = plan.instance_ranges()
                cs = torch.cumsum(torch.cat([torch.zeros(1, dtype=torch.int64, device=rc.device), rc]), 0)
                at = cs[torch.tensor(lo, device=rc.device)]
                per = (at[1:] - at[:-1]).tolist()
                return (*res, per)
            finally:
                plan.close()
        arr = self._instances(instances)
        cap = min(out_x.numel(), out_z.numel(), out_c.numel() if counts else out_x.numel())
        per = (ctypes.c_int64 * len(instances))()
        cnt = ctypes.c_int64()
        st = _stream(self.device, stream)
        if counts:
            rc = self._lib.dim3_batch_join_count(self._h, len(instances), arr, _ptr(out_x), _ptr(out_z), _ptr(out_c),
                                                 cap, per, ctypes.byref(cnt), st)
        else:
            rc = self._lib.dim3_batch_join_project(self._h, len(instances), arr, _ptr(out_x), _ptr(out_z), cap, per,
                                                   ctypes.byref(cnt), st)
        if rc == DIM3_ERR_CAPACITY:
            raise Dim3Error(rc, f"capacity {cap} < result {cnt.value}")
        _check(rc)
        n = cnt.value
        res = (out_x[:n], out_z[:n], out_c[:n]) if counts else (out_x[:n], out_z[:n])
        return (*res, list(per))

    def _join_call(self, counts, r_key, r_val, s_key, s_val, out_x, out_z, out_c, stream):
        r_key, r_val = _col(r_key, self.device, "r_key"), _col(r_val, self.device, "r_val")
        s_key, s_val = _col(s_key, self.device, "s_key"), _col(s_val, self.device, "s_val")
        cap = min(out_x.numel(), out_z.numel(), out_c.numel() if counts else out_x.numel())
        cnt = ctypes.c_int64()
        st = _stream(self.device, stream)
        if counts:
            rc = self._lib.dim3_join_count(self._h, _ptr(r_key), _ptr(r_val), r_key.numel(), _ptr(s_key),
                                           _ptr(s_val), s_key.numel(), _ptr(out_x), _ptr(out_z), _ptr(out_c), cap,
                                           ctypes.byref(cnt), st)
        else:
            rc = self._lib.dim3_join_project(self._h, _ptr(r_key), _ptr(r_val), r_key.numel(), _ptr(s_key),
                                             _ptr(s_val), s_key.numel(), _ptr(out_x), _ptr(out_z), cap,
                                             ctypes.byref(cnt), st)
        if rc == DIM3_ERR_CAPACITY:
            raise Dim3Error(rc, f"capacity {cap} < result {cnt.value}")
        _check(rc)
        n = cnt.value
        if counts:
            return out_x[:n], out_z[:n], out_c[:n]
        return out_x[:n], out_z[:n]


class ResultCache:
    """A device-resident partial result cache (Section 3)."""

    def __init__(self, ctx: Context, handle, info: CacheInfo):
        self.ctx = ctx
        self._h = handle
        self._info = info

    @property
    def info(self) -> dict:
        return {n: getattr(self._info, n) for n, _ in self._info._fields_}

    def export(self, stream=None) -> dict:
        """Entries as device tensors: z, size, complement, offsets, xs."""
        n, nl, dev = self._info.n_entries, self._info.n_list, self.ctx.device
        out = {"z": torch.empty(n, dtype=torch.int32, device=dev),
               "size": torch.empty(n, dtype=torch.int64, device=dev),
               "complement": torch.empty(n, dtype=torch.uint8, device=dev),
               "offsets": torch.empty(n + 1, dtype=torch.int64, device=dev),
               "xs": torch.empty(nl, dtype=torch.int32, device=dev)}
        _check(self.ctx._lib.dim3_cache_export(self.ctx._h, self._h, *[_ptr(out[k]) for k in
                                                                     ("z", "size", "complement", "offsets", "xs")],
                                               _stream(dev, stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            self.ctx._lib.dim3_cache_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Plan:
    """A partitioned input resident on the device (``dim3_plan``)."""

    def __init__(self, ctx: Context, handle, info: PlanInfo, stream=None, n_inst: int = 1):
        self.ctx = ctx
        self._h = handle
        self._info = info
        self.stream = stream
        self.n_inst = n_inst

    def instance_ranges(self) -> list:
        """x-id range [lo[t], lo[t+1]) of every instance of a batch plan."""
        lo = (ctypes.c_int64 * (self.n_inst + 1))()
        _check(self.ctx._lib.dim3_plan_instance_ranges(self._h, lo))
        return list(lo)

    @property
    def info(self) -> dict:
        return self._info.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self.ctx._lib.dim3_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def export(self, name: str, stream=None) -> torch.Tensor:
        which, dtype = TABLES[name]
        i = self._info
        n = {"dict_x": i.n_x, "dict_y": i.n_y, "dict_z": i.n_z, "r_rowptr": i.n_x + 1, "r_col": i.n_r_kept,
             "m_z": i.n_z, "dense_z": i.n_z, "ss_rowptr": i.n_y + 1, "ss_col": i.n_s_sparse, "deg_s": i.n_y,
             "outj_x": i.n_x}[name]
        out = torch.empty(n, dtype=dtype, device=self.ctx.device)
        _check(self.ctx._lib.dim3_plan_export(self._h, which, _ptr(out), out.numel() * out.element_size(),
                                              _stream(self.ctx.device, stream or self.stream)))
        return out

    def row_counts(self, x_begin: int = 0, x_end: int | None = None, stream=None) -> torch.Tensor:
        x_end = self._info.n_x if x_end is None else x_end
        out = torch.empty(max(x_end - x_begin, 0), dtype=torch.int64, device=self.ctx.device)
        _check(self.ctx._lib.dim3_plan_row_counts(self.ctx._h, self._h, x_begin, x_end, _ptr(out),
                                                  _stream(self.ctx.device, stream or self.stream)))
        return out

    def _run(self, counts, x_begin, x_end, out_x, out_z, out_c, stream):
        x_end = self._info.n_x if x_end is None else x_end
        L = self.ctx._lib
        st = _stream(self.ctx.device, stream or self.stream)
        cnt = ctypes.c_int64()
        if out_x is None:
            # size query (capacity 0), then allocate and emit; the plan keeps
            # the counting pass of this range, so it is not repeated
            if counts:
                rc = L.dim3_plan_join_count(self.ctx._h, self._h, x_begin, x_end, None, None, None, 0,
                                            ctypes.byref(cnt), st)
            else:
                rc = L.dim3_plan_join_project(self.ctx._h, self._h, x_begin, x_end, None, None, 0,
                                              ctypes.byref(cnt), st)
            if rc not in (DIM3_OK, DIM3_ERR_CAPACITY):
                _check(rc)
            n = cnt.value
            dev = self.ctx.device
            out_x = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            out_z = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            out_c = torch.empty(max(n, 1), dtype=torch.int32, device=dev) if counts else None
        cap = min(out_x.numel(), out_z.numel(), out_c.numel() if counts else out_x.numel())
        if counts:
            rc = L.dim3_plan_join_count(self.ctx._h, self._h, x_begin, x_end, _ptr(out_x), _ptr(out_z), _ptr(out_c),
                                        cap, ctypes.byref(cnt), st)
        else:
            rc = L.dim3_plan_join_project(self.ctx._h, self._h, x_begin, x_end, _ptr(out_x), _ptr(out_z), cap,
                                          ctypes.byref(cnt), st)
        _check(rc)
        n = cnt.value
        return (out_x[:n], out_z[:n], out_c[:n]) if counts else (out_x[:n], out_z[:n])

    def join_project(self, x_begin: int = 0, x_end: int | None = None, out_x=None, out_z=None, stream=None):
        return self._run(False, x_begin, x_end, out_x, out_z, None, stream)

    def join_count(self, x_begin: int = 0, x_end: int | None = None, out_x=None, out_z=None, out_c=None,
                   stream=None):
        return self._run(True, x_begin, x_end, out_x, out_z, out_c, stream)
