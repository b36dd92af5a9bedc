"""The classical solution on the GPU (Section 1.1: join, then deduplicate) and
the strategy choice f1 (Section 2.6), against the CPU oracle. Integer work:
bit-exact."""

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2206_04995_gb300 as dim3
from tests.gpu_util import dev, host, inst_dev

pytestmark = pytest.mark.gpu


def classical_ctx(path=dim3.PATH_CLASSICAL):
    c = dim3.Context(0)
    c.set_option(dim3.OPT_PATH, path)
    return c


def one_call(c, inst, counts=False, extra=3):
    if counts:
        ox, oz, oc, _ = oracle.join_count(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    else:
        ox, oz, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
        oc = None
    bx = torch.empty(ox.size + extra, dtype=torch.int32, device="cuda")
    bz = torch.empty(ox.size + extra, dtype=torch.int32, device="cuda")
    if counts:
        bc = torch.empty(ox.size + extra, dtype=torch.int32, device="cuda")
        x, z, cc = c.join_count(*inst_dev(inst), out_x=bx, out_z=bz, out_c=bc)
        torch.cuda.synchronize()
        assert np.array_equal(host(cc), oc.astype(np.int32))
    else:
        x, z = c.join_project(*inst_dev(inst), out_x=bx, out_z=bz)
        torch.cuda.synchronize()
    assert np.array_equal(host(x), ox) and np.array_equal(host(z), oz)


def sparse_inst(seed, n, ny, name="sparse"):
    """Uniform values: |OUT_J| about n^2 / ny."""
    rng = np.random.default_rng(seed)
    cols = [rng.integers(-10**8, 10**8, n).astype(np.int32) for _ in range(4)]
    cols[0] = rng.integers(0, ny, n).astype(np.int32)
    cols[2] = rng.integers(0, ny, n).astype(np.int32)
    return gen.Instance(name, cols[0], cols[1], cols[2], cols[3])


def _extremes():
    rng = np.random.default_rng(41)
    vals = np.array([-2**31, -2**31 + 1, -1, 0, 1, 2**31 - 2, 2**31 - 1], np.int32)
    r_key, r_val = rng.choice(vals, 300), rng.choice(vals, 300)
    s_key, s_val = rng.choice(vals, 300), rng.choice(vals, 300)
    return gen.Instance("extremes", r_key, r_val, s_key, s_val)


@pytest.mark.parametrize("counts", [False, True])
@pytest.mark.parametrize("which", ["small", "dups", "extremes", "self", "sparse", "empty_s"])
def test_classical_parity(which, counts):
    inst = {
        "small": lambda: gen.small_two_table(42, n_r=3000, n_s=2500, nx=400, ny=300, nz=350),
        "dups": lambda: gen.small_two_table(43, n_r=5000, n_s=5000, nx=50, ny=40, nz=60, dup_frac=0.3, zipf=1.2),
        "extremes": _extremes,
        "self": lambda: gen.config1_self(seed=3),
        "sparse": lambda: sparse_inst(47, 200_000, 10**6),
        "empty_s": lambda: gen.Instance("empty_s", np.arange(10, dtype=np.int32), np.arange(10, dtype=np.int32),
                                        np.zeros(0, np.int32), np.zeros(0, np.int32)),
    }[which]()
    c = classical_ctx()
    one_call(c, inst, counts)
    assert c.last_path() == dim3.PATH_CLASSICAL
    c.close()


def test_classical_capacity_short():
    inst = gen.small_two_table(44, n_r=3000, n_s=3000, nx=300, ny=200, nz=300)
    ox, _, _ = oracle.join_project(inst.r_key, inst.r_val, inst.s_key, inst.s_val)
    c = classical_ctx()
    bx = torch.empty(ox.size - 1, dtype=torch.int32, device="cuda")
    bz = torch.empty(ox.size - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(dim3.Dim3Error) as ei:
        c.join_project(*inst_dev(inst), out_x=bx, out_z=bz)
    assert ei.value.status == -4 and str(ox.size) in str(ei.value)
    c.close()


def test_f1_chooses_by_sparsity():
    """Very sparse tables (|OUT_J| close to N) take the classical path, the
    1M x 1M Zipf tables (|OUT_J| = 3500 N) the hybrid one; results agree."""
    sparse = sparse_inst(45, 500_000, 10**7)
    dense = gen.config2_two_table(scale=0.05)
    c = classical_ctx(dim3.PATH_AUTO)
    one_call(c, sparse)
    assert c.last_path() == dim3.PATH_CLASSICAL
    one_call(c, dense)
    assert c.last_path() == dim3.PATH_HYBRID
    c.close()


def test_f1_constants_steer():
    inst = gen.small_two_table(46, n_r=4000, n_s=4000, nx=500, ny=400, nz=500)
    c = classical_ctx(dim3.PATH_AUTO)
    c.set_f1_costs(1.0, 0.0, 0.0)  # mapping dear: classical
    one_call(c, inst)
    assert c.last_path() == dim3.PATH_CLASSICAL
    c.set_f1_costs(0.0, 0.0, 1.0)  # hashing dear: hybrid
    one_call(c, inst)
    assert c.last_path() == dim3.PATH_HYBRID
    with pytest.raises(dim3.Dim3Error):
        c.set_f1_costs(-1.0, 0.0, 0.0)
    c.close()
