"""Failure detection without a GPU fault: a bounded device wait whose
predecessor never publishes gives up, the call reports DIM3_ERR_TIMEOUT, and
the context keeps working."""

import numpy as np
import pytest

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import host, inst_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    ctx = dim3.Context(0)
    assert ctx.selftest_wait_timeout(0.05) == dim3.DIM3_ERR_TIMEOUT
    assert "gave up" in dim3.load().dim3_last_error().decode()
    assert ctx.selftest_wait_timeout(5.0) == dim3.DIM3_ERR_ARG  # outside (0, 2] s
    inst = gen.small_two_table(41, 4000, 4000, 400, 400, 200, zipf=1.0)
    x, z = ctx.join_project(*inst_dev(inst))
    ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)
    ctx.close()
