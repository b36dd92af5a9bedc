"""The library's deduplication-placement DP (Section 4.2, ``dim3_mjp_plan``,
host-only) against the oracle's DP: same placement, same cost. CPU only: the
library loads without a GPU and this entry point does no device work."""

import numpy as np
import pytest

import oracle

dim3 = pytest.importorskip("paper_2206_04995_gb300")


@pytest.fixture(scope="module")
def lib_ok():
    try:
        dim3.load()
    except Exception as e:  # noqa: BLE001
        pytest.skip(f"library not built: {e}")


@pytest.mark.parametrize("seed", range(30))
def test_dp_matches_oracle(lib_ok, seed):
    rng = np.random.default_rng(1000 + seed)
    k = int(rng.integers(1, 9))
    r_size = rng.integers(1, 10**7, k).astype(float).tolist()
    out_j, out_p = [r_size[0]], [r_size[0]]
    for _ in range(1, k):
        out_j.append(float(out_j[-1] * rng.uniform(0.3, 50)))
        out_p.append(float(out_j[-1] * rng.uniform(0.001, 1.0)))
    c = rng.uniform(0.0, 3.0, 5).tolist()
    dedup, cost = dim3.Context.mjp_plan(r_size, out_j, out_p, c)
    ocost, odedup = oracle.mjp_dp(r_size, out_j, out_p, c)
    assert dedup == odedup
    assert cost == pytest.approx(ocost, rel=1e-12, abs=0.0)


def test_dp_rejects_negative_costs(lib_ok):
    with pytest.raises(dim3.Dim3Error):
        dim3.Context.mjp_plan([1.0, 2.0], [1.0, 2.0], [1.0, 1.0], [1, 1, -1, 1, 1])
