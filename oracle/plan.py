"""Mapping and partition quantities of Algorithm 1, from their definitions
(test infrastructure only).

Everything is computed with numpy's sort-based ``unique`` / ``searchsorted``
and ``bincount``; no blocking or reordering beyond those definitions.

Readings of the paper used here:
* R and S are sets: duplicate input tuples collapse.
* Section 2.2, "Optimization 2": the y dictionary is built from S.y only; an
  R tuple whose y is not in S.y is dropped; S tuples are all kept.
* Section 2.2 maps every distinct value of a column to a natural number; this
  library reads "which number" as the value's rank among the column's
  distinct values (ascending, signed int32), so id order equals value order.
* Section 2.3, intersection-free partitioning: the split is made per z only;
  column z is dense when m_z >= theta_z, where m_z is the number of S tuples
  with that z (the GPU restatement of "dense if f2(z) > 0": a degree
  threshold). R is not split.
"""

from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Plan:
    dict_x: np.ndarray
    dict_y: np.ndarray
    dict_z: np.ndarray
    r_keep: np.ndarray      # bool per input R row: y in S.y
    m_x: np.ndarray         # per x id: distinct kept R tuples
    m_z: np.ndarray         # per z id: distinct S tuples
    deg_r: np.ndarray       # per y id: distinct kept R tuples
    deg_s: np.ndarray       # per y id: distinct S tuples
    out_j: int              # sum over y of deg_r * deg_s
    dense_z: np.ndarray     # bool per z id
    r_rowptr: np.ndarray    # CSR of R by x id (int64), columns = y ids ascending
    r_col: np.ndarray
    ss_rowptr: np.ndarray   # CSR of S_sparse by y id, columns = z ids ascending
    ss_col: np.ndarray


def _distinct_pairs(a: np.ndarray, b: np.ndarray):
    if a.size == 0:
        return a.astype(np.int32), b.astype(np.int32)
    packed = (a.astype(np.int64) << 32) | (b.astype(np.int64) & 0xFFFFFFFF)
    u = np.unique(packed)
    return (u >> 32).astype(np.int32), (u & 0xFFFFFFFF).astype(np.uint32).view(np.int32)


def _csr(rows: np.ndarray, cols: np.ndarray, n_rows: int):
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    rowptr = np.zeros(n_rows + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n_rows), out=rowptr[1:])
    return rowptr, cols.astype(np.int32)


def plan(r_key, r_val, s_key, s_val, theta_z: int) -> Plan:
    r_key = np.asarray(r_key, np.int32)
    r_val = np.asarray(r_val, np.int32)
    s_key = np.asarray(s_key, np.int32)
    s_val = np.asarray(s_val, np.int32)

    dict_y = np.unique(s_key)
    r_keep = np.isin(r_key, dict_y)
    rx, ry = _distinct_pairs(r_val[r_keep], r_key[r_keep])
    sz, sy = _distinct_pairs(s_val, s_key)
    dict_x = np.unique(rx)
    dict_z = np.unique(sz)

    x_id = np.searchsorted(dict_x, rx)
    ry_id = np.searchsorted(dict_y, ry)
    z_id = np.searchsorted(dict_z, sz)
    sy_id = np.searchsorted(dict_y, sy)

    m_x = np.bincount(x_id, minlength=dict_x.size).astype(np.int64)
    m_z = np.bincount(z_id, minlength=dict_z.size).astype(np.int64)
    deg_r = np.bincount(ry_id, minlength=dict_y.size).astype(np.int64)
    deg_s = np.bincount(sy_id, minlength=dict_y.size).astype(np.int64)
    out_j = int((deg_r * deg_s).sum())
    dense_z = m_z >= theta_z

    r_rowptr, r_col = _csr(x_id, ry_id, dict_x.size)
    sparse_t = ~dense_z[z_id] if z_id.size else np.zeros(0, bool)
    ss_rowptr, ss_col = _csr(sy_id[sparse_t], z_id[sparse_t], dict_y.size)

    return Plan(dict_x=dict_x, dict_y=dict_y, dict_z=dict_z, r_keep=r_keep, m_x=m_x,
                m_z=m_z, deg_r=deg_r, deg_s=deg_s, out_j=out_j, dense_z=dense_z,
                r_rowptr=r_rowptr, r_col=r_col, ss_rowptr=ss_rowptr, ss_col=ss_col)
