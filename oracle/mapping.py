"""Oracle for the mapping variants of Section 2.2 (test infrastructure only).

* ``join_project_ids`` / ``join_count_ids`` -- Optimization 1 ("skip
  mapping"): the columns already hold natural numbers (auto-increment keys,
  dictionary-encoded strings), so no mapping is done and the ids are the
  values. A negative id marks a tuple that is not part of the input (for
  instance an R tuple whose y was not found in S's dictionary, the semi-join
  of Optimization 2 done by the caller's own mapping). The result is Eq. 1
  over the remaining tuples, computed by the classical oracle.
* ``map_tuples`` -- "Supporting Wider Range of Join-Project Operations":
  several attributes are mapped together to consecutive natural numbers. Here
  the number of a tuple is its rank among the distinct tuples in
  lexicographic order (column 0 most significant; a column compares as signed
  32-bit, or as unsigned when its bit is set in ``unsigned_mask``), and the
  dictionary entry of a number is the first row holding that tuple.

Plain numpy; no blocking or reordering beyond the definitions above.
"""

from __future__ import annotations

import numpy as np

from .core import join_count, join_project


def _kept(r_y, r_x, s_y, s_z):
    r_y, r_x = np.asarray(r_y, np.int32), np.asarray(r_x, np.int32)
    s_y, s_z = np.asarray(s_y, np.int32), np.asarray(s_z, np.int32)
    kr = (r_y >= 0) & (r_x >= 0)
    ks = (s_y >= 0) & (s_z >= 0)
    return r_y[kr], r_x[kr], s_y[ks], s_z[ks]


def join_project_ids(r_y, r_x, s_y, s_z):
    """Pi_{x,z}(R join_y S) on pre-mapped ids, tuples with a negative id
    dropped. Returns (x, z, out_j) like ``join_project``."""
    return join_project(*_kept(r_y, r_x, s_y, s_z))


def join_count_ids(r_y, r_x, s_y, s_z):
    """Join-Aggregate COUNT (Section 4.1) on pre-mapped ids."""
    return join_count(*_kept(r_y, r_x, s_y, s_z))


def _sort_keys(cols, unsigned_mask):
    keys = []
    for c, col in enumerate(cols):
        a = np.asarray(col, np.int32).astype(np.int64)
        if (unsigned_mask >> c) & 1:
            a = a & 0xFFFFFFFF  # the 32 bits read as an unsigned number
        keys.append(a)
    return keys


def map_tuples(cols, unsigned_mask: int = 0):
    """(ids, first, n_distinct): ids[i] = rank of row i's tuple among the
    distinct tuples of ``cols`` (a list of k equal-length int32 columns) in
    lexicographic order; first[id] = the smallest row index with that tuple
    (array of n_distinct entries)."""
    if len(cols) == 0:
        raise ValueError("at least one column")
    keys = _sort_keys(cols, unsigned_mask)
    n = keys[0].size
    if any(k.size != n for k in keys):
        raise ValueError("column lengths differ")
    if n == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32), 0
    # np.lexsort takes the most significant key LAST and is stable, so ties
    # keep ascending row order
    order = np.lexsort(tuple(keys[::-1]))
    stacked = np.stack([k[order] for k in keys], axis=1)
    new = np.ones(n, dtype=bool)
    new[1:] = np.any(stacked[1:] != stacked[:-1], axis=1)
    rank = np.cumsum(new) - 1
    ids = np.empty(n, np.int64)
    ids[order] = rank
    first = order[new]
    return ids.astype(np.int32), first.astype(np.int32), int(new.sum())
