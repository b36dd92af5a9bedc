"""Autotuner: candidate generation and cost bounds on the CPU; on the GPU,
the chosen configuration gives the oracle's result and is cached."""

import numpy as np
import pytest

import gen
import oracle
from paper_2206_04995_gb300 import tune


def test_theta_candidates_are_degree_quantiles():
    m_z = np.array([1] * 900 + [5] * 90 + [50] * 9 + [500])
    c = tune.theta_candidates(m_z)
    assert c[0] == tune.INF
    assert 500 in c and 50 in c and 5 in c and 1 in c
    assert c == sorted(c, reverse=True)
    assert tune.theta_candidates(np.zeros(0, np.int64)) == [tune.INF]


def test_dense_estimate_bounds():
    m_z = np.array([10, 20, 30])
    n_zd, flops, b = tune.dense_estimate(m_z, 20, n_x=100, n_y=1000)
    assert n_zd == 2 and flops == 2.0 * 100 * 50 * 2
    n_zd, flops, b = tune.dense_estimate(m_z, 1, n_x=100, n_y=40)
    assert n_zd == 3 and flops == 2.0 * 100 * 40 * 3  # K bounded by |Y|
    assert tune.dense_estimate(m_z, tune.INF, 100, 40)[0] == 0


@pytest.mark.gpu
def test_tuner_decision_is_exact_and_cached(tmp_path):
    import torch

    import paper_2206_04995_gb300 as dim3
    from tests.gpu_util import host, inst_dev

    path = str(tmp_path / "tune.json")
    for inst in (gen.small_two_table(4, n_r=60_000, n_s=60_000, nx=600, ny=300, nz=500, zipf=0.7),
                 gen.config2_two_table(scale=0.02)):
        ctx = dim3.Context(0)
        cols = inst_dev(inst)
        d = tune.tune(ctx, cols, cache_path=path)
        assert not d["cached"] and d["trials"]
        x, z = ctx.join_project(*cols)
        ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
        assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
        again = tune.tune(dim3.Context(0), cols, cache_path=path)
        assert again["cached"] and again["theta"] == d["theta"] and again["variant"] == d["variant"]
        ctx.close()
        torch.cuda.synchronize()


def test_summary_counts_trials():
    tr = [{"theta": tune.INF, "variant": 0, "ms": 3.0, "n_zd": 0},
          {"theta": 9, "variant": 1, "tile_n": 256, "ms": 1.0, "n_zd": 40},
          {"theta": 9, "variant": 1, "tile_n": 128, "ms": 1.5, "n_zd": 40},
          {"theta": 4, "variant": 1, "tile_n": 256, "ms": 0.8, "n_zd": 90},
          {"theta": 9, "variant": 2, "ms": 2.0, "n_zd": 40}, {"theta": 1, "skipped": "x", "n_zd": 500}]
    d = {"theta": 4, "variant": 1, "emit_rows": 1, "ms": 0.8, "trials": tr}
    s = tune.summary(d)
    assert "trials" not in s and s["timed"] == 5 and s["skipped"] == 1 and s["theta"] == 4
    b = s["best_by_choice"]
    assert b["sparse"]["ms"] == 3.0 and b["tc256"] == {"ms": 0.8, "theta": 4, "n_zd": 90}
    assert b["tc128"]["ms"] == 1.5 and b["popc"]["ms"] == 2.0 and "probe" not in b


@pytest.mark.gpu
def test_tuner_on_a_batch_is_exact(tmp_path):
    """Tuning over a batch (timed through the batched call) leaves every
    instance's result equal to the oracle's."""
    import paper_2206_04995_gb300 as dim3
    from tests.gpu_util import host, inst_dev

    insts = gen.config4_batch(n_inst=12, lo=1000, hi=30_000)
    ctx = dim3.Context(0)
    cols = [inst_dev(i) for i in insts]
    d = tune.tune(ctx, cols, batch=True, cache_path=str(tmp_path / "t.json"))
    assert not d["cached"] and d["key"].endswith("|batch")
    x, z, per = ctx.batch_join_project(cols)
    off = np.concatenate([[0], np.cumsum(per)])
    for t, i in enumerate(insts):
        ox, oz, _ = oracle.join_project(i.r_key, i.r_val, i.s_key, i.s_val)
        assert np.array_equal(host(x[off[t]:off[t + 1]]), ox) and np.array_equal(host(z[off[t]:off[t + 1]]), oz)
    ctx.close()


def test_variant_estimates_scale_with_their_own_work():
    """The probe's bound grows with |R| and the dense index, not with |X| K:
    on a sparse-R power-law shape it stays small where the tensor-core
    operands would not fit the budget."""
    m_z = np.array([40_000] * 200 + [10] * 200_000)
    est = tune.variant_estimates(m_z, 1000, n_x=220_000, n_y=220_000, n_r=2_000_000)
    tc_s, tc_b = est[tune.dim3.DENSE_TC]
    pr_s, pr_b = est[tune.dim3.DENSE_PROBE]
    po_s, po_b = est[tune.dim3.DENSE_POPC]
    assert tc_b > tune.DENSE_BYTES_BUDGET > pr_b and pr_s < tc_s and pr_s < po_s
    assert tune.variant_estimates(m_z, 10**9, 1, 1, 1) == {}
