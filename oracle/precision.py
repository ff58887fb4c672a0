"""Reduced-precision storage of the sparse inverse and the residual correction.

TEST INFRASTRUCTURE (see the package docstring). Not a method of the paper: the paper
stores S~ in the working precision. This module states in FP64 what a solver computes when
the values of S~ = L~^-1 P (Eq. 7, Theorem 1) are stored rounded to BF16 and products run
in exact arithmetic, and what one residual correction x <- x + S^T S (b - A x) then
computes. Both sides round in the same way: the FP64 value to the nearest FP32 value, that
to the nearest BF16 value, ties to even each time.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def bf16_round(x):
    """FP64 array -> FP64 array of the nearest BF16 values of its FP32 roundings (ties to
    even). BF16 keeps the FP32 sign, the 8-bit exponent and the top 7 stored mantissa bits,
    so rounding the FP32 bit pattern at bit 16 gives the nearest BF16 number."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def sparse_inverse_dense(A, perm):
    """S = L^-1 P as a dense matrix, with P A P^T = L L^T and (P x)_k = x[perm[k]], so that
    S^T S = A^-1 (Eq. 7). Dense: for the small meshes of the tests."""
    A = np.asarray(A, dtype=np.float64)
    perm = np.asarray(perm)
    L = np.linalg.cholesky(A[np.ix_(perm, perm)])
    Linv = sla.solve_triangular(L, np.eye(len(perm)), lower=True)
    return Linv


def apply_rounded_inverse(Linv_r, perm, b):
    """x = S^T (S b) with the (rounded) values Linv_r of S = L^-1 P; b: n x k."""
    b = np.asarray(b, dtype=np.float64)
    z = Linv_r @ b[perm]
    x = np.empty_like(b)
    x[perm] = Linv_r.T @ z
    return x


def solve_bf16(A, perm, b, corrections):
    """The global solve with BF16 values of S and `corrections` residual corrections
    x <- x + S^T S (b - A x), all arithmetic exact (FP64). Returns the list of iterates
    [x_0, ..., x_corrections]."""
    Sr = bf16_round(sparse_inverse_dense(A, perm))
    xs = [apply_rounded_inverse(Sr, perm, b)]
    for _ in range(corrections):
        r = b - np.asarray(A) @ xs[-1]
        xs.append(xs[-1] + apply_rounded_inverse(Sr, perm, r))
    return xs
