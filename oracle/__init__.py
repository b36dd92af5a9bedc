"""CPU oracle for the DIM^3 Join-Project hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(the CUDA library and its binding) never imports, links or runs it, and it
shares no code with that path.

* ``join_project`` / ``join_count`` -- Eq. 1 (Section 1) computed by the
  classical solution (Section 1.1): hash join on y, hash-based duplicate
  elimination, sort (``oracle.c``).
* ``rank_map`` -- the order-preserving value mapping (Section 2.2).
* ``join_project_ids`` / ``join_count_ids`` / ``map_tuples`` -- Section 2.2's
  skipped mapping (Optimization 1) and multi-attribute mapping
  (``mapping.py``).
* ``cache_stats`` / ``cache_select`` / ``cache_build`` /
  ``join_project_cached`` -- partial result caching, Section 3 (``cache.py``).
* ``join_aggregate`` / ``groupby_aggregate`` -- Join-Aggregate, Section 4.1,
  from the materialised join (``aggregate.py``).
* ``line_join_project`` / ``chain_sizes`` / ``mjp_dp`` -- multi-way joins
  with projection and the deduplication-placement DP, Section 4.2 (``mjp.py``).
* ``plan`` -- the mapping and partition quantities of Algorithm 1 (semi-join
  filtered y dictionary of Section 2.2 "Optimization 2", x/z dictionaries,
  degrees m_x and m_z, |OUT_J|, the dense z set of Section 2.3) written out
  from their definitions with numpy (``plan.py``).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, a library boolean matmul, the paper's textual examples, closed
forms and invariants).
"""

from .core import (  # noqa: F401
    build,
    join_count,
    join_project,
    lib_path,
    rank_map,
)
from .aggregate import groupby_aggregate, join_aggregate  # noqa: F401
from .cache import cache_build, cache_scores, cache_select, cache_stats, join_project_cached  # noqa: F401
from .mjp import chain_sizes, line_join_project  # noqa: F401
from .mjp import dp as mjp_dp  # noqa: F401
from .mapping import join_count_ids, join_project_ids, map_tuples  # noqa: F401
from .plan import plan  # noqa: F401
