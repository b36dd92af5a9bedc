"""Seeded synthetic inputs for the DIM^3 Join-Project path.

This package holds random draws and input-tuple deduplication only. It
contains none of the method's arithmetic, so both the CPU oracle's tests and
the CUDA path can consume the same arrays.
"""

from .synth import (  # noqa: F401
    CONFIGS,
    Instance,
    chung_lu_self,
    chung_lu_uncapped,
    config1_self,
    config2_two_table,
    config3_chung_lu,
    config4_batch,
    config5_stream,
    random_ids,
    small_two_table,
    two_table,
    zipf_ranks,
)
