"""The persistent pipelined emitting kernel (DIM3_OPT_EMIT_PIPELINE: a CTA
publishes a row group's pair count, builds the next group, then resolves and
writes the first) against the oracle: single instances and batches, output
buffers at unaligned offsets, a capacity that is too short, and the row
counts it leaves for later queries."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import host, inst_dev

pytestmark = pytest.mark.gpu


def ctx_pipe(extra=None):
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, dim3.PATH_HYBRID)
    c.set_option(dim3.OPT_EMIT_PIPELINE, 1)
    for k, v in (extra or {}).items():
        c.set_option(k, v)
    return c


INSTS = {
    "zipf_0.05": lambda: gen.config2_two_table(scale=0.05),
    "zipf_0.02": lambda: gen.config2_two_table(scale=0.02),
    "small_dups": lambda: gen.small_two_table(5, n_r=9000, n_s=7000, nx=901, ny=300, nz=700, zipf=1.0, dup_frac=0.1),
    "self": lambda: gen.config1_self(),
    "one_row": lambda: gen.small_two_table(6, n_r=50, n_s=400, nx=1, ny=20, nz=90),
}


@pytest.mark.parametrize("name", list(INSTS))
def test_pipe_vs_oracle(name):
    inst = INSTS[name]()
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    for opts in ({}, {dim3.OPT_BITMAP_ROW_MIN: 1}, {dim3.OPT_THETA_Z: 6, dim3.OPT_DENSE_VARIANT: dim3.DENSE_TC}):
        c = ctx_pipe(opts)
        try:
            bx = torch.empty(ox.size + 9, dtype=torch.int32, device="cuda")
            bz = torch.empty(ox.size + 9, dtype=torch.int32, device="cuda")
            x, z = c.join_project(*inst_dev(inst), out_x=bx[1:], out_z=bz[3:])
            assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz), (name, opts)
        finally:
            c.close()


def test_pipe_row_counts_and_capacity():
    inst = gen.config2_two_table(scale=0.02)
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    c = ctx_pipe()
    try:
        cols = inst_dev(inst)
        plan = c.partition(*cols)
        bx = torch.empty(ox.size, dtype=torch.int32, device="cuda")
        bz = torch.empty(ox.size, dtype=torch.int32, device="cuda")
        x, z = plan.join_project(out_x=bx, out_z=bz)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        # the counts recorded by the single pass answer the row-count query
        dx = host(plan.export("dict_x"))
        rc = host(plan.row_counts())
        ux, cnt = np.unique(ox, return_counts=True)
        exp = np.zeros(dx.size, np.int64)
        exp[np.searchsorted(dx, ux)] = cnt
        assert np.array_equal(rc, exp)
        plan.close()
        with pytest.raises(dim3.Dim3Error) as ei:
            c.join_project(*cols, out_x=bx[: ox.size // 3], out_z=bz[: ox.size // 3])
        assert ei.value.status == dim3.DIM3_ERR_CAPACITY and str(ox.size) in str(ei.value)
    finally:
        c.close()


def test_pipe_batch():
    insts = gen.config4_batch(n_inst=9, lo=1000, hi=20_000) + [gen.small_two_table(7, n_r=0, n_s=10, nx=3, ny=3, nz=3)]
    c = ctx_pipe({dim3.OPT_EMIT_ROWS: 2})
    try:
        x, z, per = c.batch_join_project([inst_dev(i) for i in insts])
        off = np.concatenate([[0], np.cumsum(per)])
        for t, i in enumerate(insts):
            ox, oz, _ = oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)
            assert np.array_equal(host(x[off[t]:off[t + 1]]), ox) and np.array_equal(host(z[off[t]:off[t + 1]]), oz)
    finally:
        c.close()
