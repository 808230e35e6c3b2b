"""Maximum-product matching and scaling (the role MC64 plays in §2, Eq. mc64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

§2 asks for a row permutation and scalings, Abar = P D_r A D_c, that put entries of
modulus one on the diagonal and leave every other entry of modulus at most one;
the paper uses HSL MC64 for it.  MC64 is not available, so this restates the
standard formulation behind it:

  cost  c_ij = log(max_k |a_kj|) - log|a_ij| >= 0   for every nonzero a_ij,
  a perfect matching sigma (row sigma(j) for column j) of minimum total cost,
  i.e. maximum product of |a_{sigma(j) j}|, and dual variables u (rows), v
  (columns) with u_i + v_j <= c_ij on every nonzero and equality on the matching.

Then D_r = exp(u), D_c = exp(v) / colmax satisfy |d_r,i a_ij d_c,j| =
exp(u_i + v_j - c_ij) <= 1, with equality on the matched entries, which the
permutation (row j of Abar = row sigma(j)) moves to the diagonal.

The matching and the duals come from successive shortest augmenting paths
(Dijkstra on reduced costs c_ij - u_i - v_j, the Hungarian method for sparse
bipartite graphs), one augmentation per row.
"""
from __future__ import annotations

import heapq

import numpy as np
import scipy.sparse as sp


def matching_costs(A):
    """(CSR of costs c_ij on A's pattern, column maxima)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    absA = abs(A)
    colmax = np.asarray(absA.max(axis=0).todense()).ravel()
    if np.any(colmax == 0):
        raise ValueError("A has an empty column")
    C = absA.copy()
    C.data = np.log(colmax[C.indices]) - np.log(C.data)
    return C, colmax


def max_product_matching(A):
    """Minimum-cost perfect matching on the costs above, with its duals.

    Returns (row_of_col, u, v, total_cost); raises ValueError when A is
    structurally singular (no perfect matching)."""
    C, _ = matching_costs(A)
    n = C.shape[0]
    indptr, indices, cost = C.indptr, C.indices, C.data
    u = np.zeros(n)
    v = np.zeros(n)
    row_of_col = np.full(n, -1, dtype=np.int64)
    col_of_row = np.full(n, -1, dtype=np.int64)
    for s in range(n):
        # Dijkstra from the free row s; nodes: rows and columns
        dist_c = np.full(n, np.inf)
        pred_c = np.full(n, -1, dtype=np.int64)       # row from which column j was reached
        dist_r = {s: 0.0}
        done_c = np.zeros(n, dtype=bool)
        popped_rows = []
        popped_cols = []
        heap = [(0.0, 0, s)]                           # (dist, kind 0 = row / 1 = column, index)
        sink, D = -1, np.inf
        while heap:
            d, kind, x = heapq.heappop(heap)
            if kind == 0:
                if d > dist_r.get(x, np.inf):
                    continue
                popped_rows.append(x)
                for e in range(indptr[x], indptr[x + 1]):
                    j = indices[e]
                    if done_c[j]:
                        continue
                    nd = d + (cost[e] - u[x] - v[j])
                    if nd < dist_c[j]:
                        dist_c[j] = nd
                        pred_c[j] = x
                        heapq.heappush(heap, (nd, 1, j))
            else:
                if done_c[x] or d > dist_c[x]:
                    continue
                done_c[x] = True
                popped_cols.append(x)
                if row_of_col[x] < 0:
                    sink, D = x, d
                    break
                i2 = row_of_col[x]                      # matched edge, reduced cost 0
                if d < dist_r.get(i2, np.inf):
                    dist_r[i2] = d
                    heapq.heappush(heap, (d, 0, i2))
        if sink < 0:
            raise ValueError("A is structurally singular: no perfect matching")
        for i in popped_rows:
            u[i] += D - dist_r[i]
        for j in popped_cols:
            v[j] -= D - dist_c[j]
        j = sink                                        # augment along the predecessors
        while True:
            i = pred_c[j]
            jn = col_of_row[i]
            row_of_col[j] = i
            col_of_row[i] = j
            if i == s:
                break
            j = jn
    total = 0.0
    for j in range(n):
        i = row_of_col[j]
        e = indptr[i] + np.searchsorted(indices[indptr[i]:indptr[i + 1]], j)
        total += cost[e]
    return row_of_col, u, v, total


def matching_scaling(A):
    """(row_perm, dr, dc) of Eq. mc64 from the matching: row i of Abar is row
    row_perm[i] of D_r A D_c, |diag(Abar)| = 1 and |Abar_ij| <= 1."""
    _, colmax = matching_costs(A)
    row_of_col, u, v, _ = max_product_matching(A)
    return row_of_col.copy(), np.exp(u), np.exp(v) / colmax
