"""Planted mistakes in the oracle must be caught by the pins.

Each case compiles a copy of ``oracle/oracle.c`` with one plausible mistake
(a swapped operand, a missed dedup, a wrong sign convention, a dropped join
tuple, an off-by-one rank) into a temporary library, swaps it in, and checks
that at least one pin from ``test_oracle_pins`` fails. The real oracle is
restored afterwards. CPU only.
"""

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import oracle.core as core
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTATIONS = {
    "swap_x_z": ("pack(r_val[i], s_val[j])", "pack(s_val[j], r_val[i])"),
    "no_input_dedup": ("if (!ins) continue; /* duplicate R tuple */", "(void)ins;"),
    "unsigned_order": ("return packed_xz ^ 0x8000000080000000ULL;", "return packed_xz;"),
    "skip_first_chain_tuple": ("for (int64_t j = head[ybucket.vals[s]]; j >= 0; j = next[j])",
                               "for (int64_t j = next[head[ybucket.vals[s]]]; j >= 0; j = next[j])"),
    "rank_off_by_one": ("if (sorted[mid] < vals[i]) lo = mid + 1;",
                        "if (sorted[mid] <= vals[i]) lo = mid + 1;"),
}


def _pins():
    yield lambda: [pins.test_bruteforce_tiny(s) for s in range(24)]
    yield lambda: [pins.test_shuffle_and_duplicate_invariance(s) for s in range(4)]
    yield pins.test_canonical_signed_order
    yield lambda: [pins.test_rank_map_against_unique(s) for s in range(5)]
    yield pins.test_fig3_single_emission


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "libm.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", c, "-o", so])
        core._load()  # make sure the real library is set up first
        real = core._lib
        mutant = ctypes.CDLL(so)
        for fn in ("oracle_join", "oracle_result_size", "oracle_result_out_j",
                   "oracle_result_copy", "oracle_result_free", "oracle_rank_map"):
            getattr(mutant, fn).restype = getattr(real, fn).restype
            getattr(mutant, fn).argtypes = getattr(real, fn).argtypes
        monkeypatch.setattr(core, "_lib", mutant)
        caught = 0
        for pin in _pins():
            try:
                pin()
            except (AssertionError, IndexError, ValueError):
                caught += 1
        assert caught >= 1, f"no pin caught mutation {name}"
    # the real oracle still passes
    monkeypatch.setattr(core, "_lib", real)
    pins.test_bruteforce_tiny(0)
    assert np.array_equal(oracle.rank_map(np.array([3, 1, 3], np.int32))[0], [1, 0, 1])
