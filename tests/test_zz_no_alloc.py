"""dim3_map_noalloc, the mapping entry point for callers that may not allocate
device memory, against dim3_map and against the oracle's rank map (exact
equality), on calls in a row.

The second call is smaller than the first and reuses the same fixed scratch
array, so a result that leaned on leftovers of the first call would show
here. Collected last so that a stop at the first failure has run every other
test already; passes alone in a fresh process as well.
"""

import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3

pytestmark = pytest.mark.gpu

MAX_N = 1 << 16


def _fn():
    lib = dim3.load()
    f = lib.dim3_map_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return lib, f


def _map_noalloc(vals: torch.Tensor):
    lib, f = _fn()
    n = vals.numel()
    ids = torch.full((max(n, 1),), -123, dtype=torch.int32, device=vals.device)
    dct = torch.full((max(n, 1),), -123, dtype=torch.int32, device=vals.device)
    nd = ctypes.c_int64(-1)
    rc = f(ctypes.c_void_p(vals.data_ptr()), n, ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dct.data_ptr()),
           ctypes.byref(nd), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, ids[:n], dct[: max(nd.value, 0)], nd.value, lib


def _columns():
    """Value columns in call order: the largest column, a smaller one
    after it, a table filled to its largest load (65,536 distinct values in
    131,072 slots) and a short column of INT32 extremes, 0 and -1 with
    repeats (the order of the signed sort key)."""
    out = []
    for n, pool, seed in [(MAX_N, 40_000, 1), (9_000, 1_500, 2)]:
        rng = np.random.default_rng(seed)
        out.append(gen.random_ids(rng, pool)[rng.integers(0, pool, size=n)])
    out.append(gen.random_ids(np.random.default_rng(3), MAX_N))
    ext = np.array([2**31 - 1, -2**31, 0, -1, 1, -2**31, 2**31 - 1, 0, -1, -2, 2**31 - 2, -2**31 + 1] * 5,
                   dtype=np.int64).astype(np.int32)
    out.append(np.random.default_rng(4).permutation(ext))
    return out


def test_map_noalloc_matches_map_and_oracle_on_calls_in_a_row():
    ctx = dim3.Context(0)
    try:
        for vals in _columns():
            d_vals = torch.from_numpy(np.ascontiguousarray(vals, np.int32)).cuda()
            ref_ids, ref_dict = ctx.map(d_vals)
            rc, ids, dct, nd, lib = _map_noalloc(d_vals)
            assert rc == 0, lib.dim3_last_error()
            torch.cuda.synchronize()
            assert nd == ref_dict.numel()
            assert torch.equal(ids, ref_ids)
            assert torch.equal(dct, ref_dict)
            o_ids, o_dict = oracle.rank_map(vals)
            assert np.array_equal(ids.cpu().numpy(), o_ids)
            assert np.array_equal(dct.cpu().numpy(), o_dict)
    finally:
        ctx.close()


def test_map_noalloc_rejects_oversize_column():
    d_vals = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    rc, _, _, _, lib = _map_noalloc(d_vals)
    assert rc == -6  # DIM3_ERR_OVERFLOW
    assert b"65536" in lib.dim3_last_error()
