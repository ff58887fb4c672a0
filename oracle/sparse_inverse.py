"""Elimination tree, Cholesky factor and its sparse inverse S = L^-1 (Sec. 4.2, Theorem 1,
Alg. 2; Eq. 7: A^-1 = S^T S).

TEST INFRASTRUCTURE (see the package docstring). Plain FP64, dense arithmetic for small
matrices; used to pin the structure theorem and the identity A^-1 = S^T S, not on the
frame loop (which uses the plain definition A^-1 b).

With a symmetric permutation P (PAP^T = L L^T) the sparse inverse is S = L^-1 P, so that
S^T S = P^T L^-T L^-1 P = A^-1 holds for the unpermuted A.
"""
from __future__ import annotations

import numpy as np


def etree(A):
    """Elimination tree of a symmetric matrix (dense or scipy sparse): parent[j] is the
    smallest i > j with L[i, j] != 0 structurally, -1 for a root. Computed by the
    path-compressed ancestor walk over the lower triangle, row by row."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    n = A.shape[0]
    parent = -np.ones(n, dtype=np.int64)
    ancestor = -np.ones(n, dtype=np.int64)
    for k in range(n):
        cols = A.indices[A.indptr[k]:A.indptr[k + 1]]
        for j in cols[cols < k]:
            i = j
            while i != -1 and i < k:
                nxt = ancestor[i]
                ancestor[i] = k
                if nxt == -1:
                    parent[i] = k
                i = nxt
    return parent


def ancestors(parent, j):
    """j and all its ancestors, in increasing order."""
    out = []
    while j != -1:
        out.append(j)
        j = parent[j]
    return out


def ancestor_closure_pattern(parent):
    """Boolean n x n matrix with (i, j) set iff i is j or an ancestor of j (Theorem 1)."""
    n = len(parent)
    P = np.zeros((n, n), dtype=bool)
    for j in range(n):
        P[ancestors(parent, j), j] = True
    return P


def postorder(parent):
    """A postorder of the forest (children before parents, subtrees contiguous)."""
    n = len(parent)
    children = [[] for _ in range(n)]
    roots = []
    for j in range(n):
        (children[parent[j]] if parent[j] >= 0 else roots).append(j)
    order = []
    for r in roots:
        stack = [(r, 0)]
        while stack:
            v, i = stack.pop()
            if i < len(children[v]):
                stack.append((v, i + 1))
                stack.append((children[v][i], 0))
            else:
                order.append(v)
    return np.array(order, dtype=np.int64)


def cholesky(A):
    """Dense lower Cholesky factor (numpy), A = L L^T."""
    return np.linalg.cholesky(np.asarray(A, dtype=np.float64))


def sparse_inverse_columns(L, parent):
    """S = L^-1 built one column at a time (Alg. 2, second line; Sec. 4.2 figure): column j
    solves L x = e_j, and x is non-zero only on j and its elimination-tree ancestors, so the
    forward substitution visits only those rows."""
    n = L.shape[0]
    S = np.zeros((n, n))
    for j in range(n):
        path = ancestors(parent, j)
        x = np.zeros(n)
        x[j] = 1.0
        for a in path:
            x[a] /= L[a, a]
            below = [r for r in path if r > a]
            x[below] -= L[below, a] * x[a]
        S[path, j] = x[path]
    return S
