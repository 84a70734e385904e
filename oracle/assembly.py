"""Assembly oracle -- TEST INFRASTRUCTURE ONLY (the rules of ``oracle``
apply: only the tests, ``smoke()`` and the bench's CPU baseline use it).

* ``assemble`` -- Sec. 2: entry (r, c) of the global matrix is the sum of
  the element entries A_e[i][j] whose local functions carry the global
  numbers r = l2g_e[i] and c = l2g_e[j], and the global load vector gathers
  b_e[i] at l2g_e[i].  Written out with numpy in element order: every
  element entry is keyed by (r, c), the distinct keys sorted by row and
  column form the CSR pattern, and np.add.at sums the entries into them.
* ``assemble_dense`` -- the same sum as an explicit loop into a dense
  matrix, for tiny inputs (a second, independent statement of the sum).
"""
from __future__ import annotations

import numpy as np


def _offsets(degrees):
    p = np.asarray(degrees, dtype=np.int64)
    s = (p + 1) ** 2 * (p + 2) // 2
    loff = np.concatenate([[0], np.cumsum(s)])
    moff = np.concatenate([[0], np.cumsum(s * s)])
    return s, loff, moff


def assemble(A, bvec, l2g, n_dof, degrees):
    """CSR assembly of element matrices A (flat, element e's N_sh x N_sh
    row-major block at sum of N_sh^2 over earlier elements) and vectors
    bvec (flat, at sum of N_sh) with the map l2g (flat like bvec).
    Returns row_ptr int64 [n_dof + 1], col_idx int32 [nnz], values float64
    [nnz] and rhs float64 [n_dof]."""
    s, loff, moff = _offsets(degrees)
    rows, cols = [], []
    for e in range(len(s)):
        g = np.asarray(l2g[loff[e]:loff[e + 1]], dtype=np.int64)
        rows.append(np.repeat(g, s[e]))
        cols.append(np.tile(g, s[e]))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    key = r * n_dof + c
    ukey, inv = np.unique(key, return_inverse=True)
    values = np.zeros(len(ukey))
    np.add.at(values, inv, np.asarray(A, dtype=np.float64)[:moff[-1]])
    urow = ukey // n_dof
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(urow, minlength=n_dof))]).astype(np.int64)
    col_idx = (ukey % n_dof).astype(np.int32)
    rhs = np.zeros(n_dof)
    np.add.at(rhs, np.asarray(l2g, dtype=np.int64)[:loff[-1]], np.asarray(bvec, dtype=np.float64)[:loff[-1]])
    return row_ptr, col_idx, values, rhs


def assemble_dense(A, bvec, l2g, n_dof, degrees):
    """Dense K [n_dof, n_dof] and rhs by a plain triple loop (tiny inputs)."""
    s, loff, moff = _offsets(degrees)
    K = np.zeros((n_dof, n_dof))
    rhs = np.zeros(n_dof)
    for e in range(len(s)):
        for i in range(s[e]):
            r = int(l2g[loff[e] + i])
            rhs[r] += bvec[loff[e] + i]
            for j in range(s[e]):
                K[r, int(l2g[loff[e] + j])] += A[moff[e] + i * s[e] + j]
    return K, rhs


def csr_to_dense(row_ptr, col_idx, values, n_dof):
    K = np.zeros((n_dof, n_dof))
    for r in range(n_dof):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            K[r, col_idx[k]] += values[k]
    return K
