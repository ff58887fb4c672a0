"""Pins of the reduced-precision oracle: BF16 rounding against a brute-force nearest-value
search on the BF16 grid, the sparse inverse against A^-1, and the correction against the
exact error recursion e_1 = (I - M A) e_0 with M = S^T S."""
import math

import numpy as np
import pytest

from oracle.precision import (apply_rounded_inverse, bf16_round, solve_bf16,
                              sparse_inverse_dense)


def _bf16_neighbours(v):
    """The two BF16 numbers around the FP32 value v (|v| normal), from frexp: BF16 has 8
    significant bits, so its spacing on [2^(e-1), 2^e) is 2^(e-8)."""
    m, e = math.frexp(abs(v))
    step = 2.0 ** (e - 8)
    lo = math.floor(abs(v) / step) * step
    return math.copysign(lo, v), math.copysign(lo + step, v), step


def test_bf16_round_is_the_nearest_value_ties_to_even():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.normal(size=4000) * 10.0 ** rng.integers(-20, 20, 4000),
                           rng.uniform(-1, 1, 1000)])
    r = bf16_round(vals)
    for v, got in zip(vals.astype(np.float32).astype(np.float64), r):
        a, b, step = _bf16_neighbours(v)
        da, db = abs(v - a), abs(v - b)
        if da < db:
            assert got == a
        elif db < da:
            assert got == b
        else:  # tie: the even one has an even multiple of the step
            want = a if round(abs(a) / step) % 2 == 0 else b
            assert got == want


def test_bf16_round_special_cases():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1.0);
    # 1 + 3 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: the even one is 1 + 2^-6
    x = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -2.5, 0.0, 3.0e38 * 10])
    with np.errstate(over="ignore"):
        r = bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2.0 ** -6 and r[3] == -2.5
    assert r[4] == 0.0 and np.isinf(r[5])
    assert np.array_equal(bf16_round(r[:5]), r[:5])            # idempotent
    y = np.sort(np.random.default_rng(1).normal(size=2000))
    assert np.all(np.diff(bf16_round(y)) >= 0)                 # monotone
    rel = np.abs(bf16_round(y) - y) / np.abs(y)
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)                  # half a unit in the last place


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, n))
    return B @ B.T + n * np.eye(n)


def test_sparse_inverse_dense_gives_the_inverse():
    A = _spd(30, 2)
    perm = np.random.default_rng(3).permutation(30)
    S = sparse_inverse_dense(A, perm)
    assert np.allclose(np.tril(S), S)
    P = np.eye(30)[perm]
    assert np.allclose((S @ P).T @ (S @ P) @ A, np.eye(30), atol=1e-10)
    b = np.random.default_rng(4).normal(size=(30, 3))
    assert np.allclose(apply_rounded_inverse(S, perm, b), np.linalg.solve(A, b), atol=1e-10)


def test_bf16_solve_error_and_correction_recursion():
    A = _spd(40, 5)
    perm = np.arange(40)[::-1].copy()
    b = np.random.default_rng(6).normal(size=(40, 3))
    xs = solve_bf16(A, perm, b, corrections=2)
    x = np.linalg.solve(A, b)
    S = bf16_round(sparse_inverse_dense(A, perm))
    P = np.eye(40)[perm]
    M = (S @ P).T @ (S @ P)
    e0, e1, e2 = (xi - x for xi in xs)
    # one correction maps the error through I - M A (exact recursion)
    assert np.allclose(e1, (np.eye(40) - M @ A) @ e0, atol=1e-12 * np.abs(x).max())
    assert np.allclose(e2, (np.eye(40) - M @ A) @ e1, atol=1e-12 * np.abs(x).max())
    # BF16 storage: the plain solve is off by O(2^-8); this matrix is well conditioned,
    # so the correction contracts the error
    rel = [np.linalg.norm(e) / np.linalg.norm(x) for e in (e0, e1, e2)]
    assert 1e-5 < rel[0] < 2e-2
    assert rel[1] < 0.1 * rel[0] and rel[2] < 0.1 * rel[1]
