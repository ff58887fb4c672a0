"""Pins of Theorem 1 (the pattern of L^-1 is the elimination-tree ancestor closure) and of
A^-1 = S^T S with S = L^-1 P (Eq. 7), on small SPD matrices built from tetrahedral meshes."""
import numpy as np
import scipy.sparse as sp

import scenegen as sg
from oracle import sparse_inverse as SI
from oracle.fem import FEM


def _scalar_matrix(m=4, seed=0):
    """A per-vertex SPD matrix with the mesh's connectivity and generic values."""
    sc = sg.cube_drop(m=m, seed=seed)
    n = sc.n_verts
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for t in sc.tets:
        for a in t:
            for b in t:
                rows.append(a)
                cols.append(b)
    P = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    P.data[:] = 1.0
    vals = -rng.uniform(0.1, 1.0, P.nnz)
    A = sp.csr_matrix((vals, P.indices.copy(), P.indptr.copy()), shape=(n, n)).toarray()
    A = 0.5 * (A + A.T)
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(A, -A.sum(1) + rng.uniform(0.5, 1.0, n))
    return A


def test_etree_matches_structure_of_numeric_factor():
    A = _scalar_matrix()
    L = SI.cholesky(A)
    parent = SI.etree(A)
    n = len(A)
    for j in range(n):
        below = np.nonzero(np.abs(L[j + 1:, j]) > 1e-14)[0]
        expect = j + 1 + below[0] if len(below) else -1
        assert parent[j] == expect


def test_theorem1_pattern_is_ancestor_closure():
    for seed, perm_seed in [(0, None), (1, 5), (2, 9)]:
        A = _scalar_matrix(seed=seed)
        if perm_seed is not None:
            p = np.random.default_rng(perm_seed).permutation(len(A))
            A = A[np.ix_(p, p)]
        L = SI.cholesky(A)
        Linv = np.linalg.inv(L)
        parent = SI.etree(A)
        pattern = np.abs(Linv) > 1e-13 * np.abs(Linv).max()
        closure = SI.ancestor_closure_pattern(parent)
        assert not np.any(pattern & ~closure)          # no entry outside the closure
        assert np.array_equal(pattern, closure)         # generic values: all of it filled


def test_sparse_inverse_by_ancestor_columns_equals_dense_inverse():
    A = _scalar_matrix(seed=3)
    L = SI.cholesky(A)
    S = SI.sparse_inverse_columns(L, SI.etree(A))
    assert np.abs(S - np.linalg.inv(L)).max() < 1e-12 * np.abs(S).max()
    assert np.abs(S.T @ S - np.linalg.inv(A)).max() < 1e-10 * np.abs(np.linalg.inv(A)).max()


def test_postorder_makes_rows_contiguous_profiles():
    A = _scalar_matrix(seed=4)
    po = SI.postorder(SI.etree(A))
    Ap = A[np.ix_(po, po)]
    parent = SI.etree(Ap)
    assert np.all((parent == -1) | (parent > np.arange(len(parent))))
    Linv = np.linalg.inv(SI.cholesky(Ap))
    for i in range(len(Ap)):
        nz = np.nonzero(np.abs(Linv[i]) > 1e-13 * np.abs(Linv).max())[0]
        assert nz[-1] == i and np.array_equal(nz, np.arange(nz[0], i + 1))


def test_sparse_inverse_solves_the_pd_system():
    # the full 3n system of a small cube: S^T S b equals the direct solve, with S = L^-1 P
    sc = sg.cube_drop(m=3)
    fem = FEM(sc)
    A = fem.A_ff.toarray()
    p = SI.postorder(SI.etree(A))
    Ap = A[np.ix_(p, p)]
    L = SI.cholesky(Ap)
    Sp = SI.sparse_inverse_columns(L, SI.etree(Ap))
    S = Sp[:, np.argsort(p)]                      # S = L^-1 P
    b = np.random.default_rng(0).normal(size=len(A))
    x = S.T @ (S @ b)
    assert np.abs(x - fem.solve(b)).max() < 1e-11 * np.abs(x).max()
