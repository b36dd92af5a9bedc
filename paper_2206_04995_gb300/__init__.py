"""GB300-native (sm_103a) DIM^3 Join-Project.

The hot path of DIM^3 (value mapping, intersection-free dense/sparse split,
SparseBMM, DenseEC, compaction of the deduplicated (x, z) output) runs in the
CUDA library ``libdim3.so`` behind the C ABI of ``include/dim3.h``; this
package is its thin binding (``dim3``), plus the batch runner, the serving
loop and the autotuner built on that ABI.
"""

from .dim3 import (  # noqa: F401
    AGG_AVG,
    AGG_COUNT,
    AGG_MAX,
    AGG_MIN,
    AGG_SUM,
    DIM3_ERR_ARG,
    DIM3_ERR_CAPACITY,
    DIM3_ERR_CUDA,
    DIM3_ERR_NOMEM,
    DIM3_ERR_OVERFLOW,
    DIM3_ERR_TIMEOUT,
    DIM3_ERR_UNSUPPORTED,
    DIM3_OK,
    DENSE_AUTO,
    DENSE_POPC,
    DENSE_PROBE,
    DENSE_TC,
    FN_ADD,
    FN_LEFT,
    FN_MUL,
    FN_RIGHT,
    OPT_BITMAP_ROW_MIN,
    OPT_DENSE_VARIANT,
    OPT_EMIT_ROWS,
    OPT_ID_CHUNK_MAX,
    OPT_LIGHT_ROW_MAX,
    OPT_PATH,
    OPT_TILE_WORDS,
    OPT_DENSE_TILE_N,
    PATH_AUTO,
    PATH_CLASSICAL,
    PATH_HYBRID,
    OPT_THETA_Z,
    OPT_TIMING,
    OPT_TWO_PASS,
    PHASES,
    Context,
    Dim3Error,
    Plan,
    ResultCache,
    launch_count,
    lib_path,
    load,
)
