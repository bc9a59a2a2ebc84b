"""Pins for the oracle's half-stored symmetric SpMM (Sec. 3.1: half-stored H)."""
import numpy as np
import pytest

import oracle as O
from gen import ci_matrix, laplacian_kron, laplacian_kron_eigs, CSRUpper


def dense_by_loops(H):
    """Expand the stored upper triangle entry by entry (independent of scipy)."""
    A = np.zeros((H.n, H.n))
    v = H.values_f64()
    for i in range(H.n):
        for k in range(H.rowptr[i], H.rowptr[i + 1]):
            j = int(H.col[k])
            A[i, j] = v[k]
            A[j, i] = v[k]
    return A


def lap_eigvec(dims, ks):
    """Closed-form eigenvector of the Kronecker-sum Laplacian: product of sines."""
    grids = np.meshgrid(*[np.sin(np.pi * k * np.arange(1, m + 1) / (m + 1)) for m, k in zip(dims, ks)],
                        indexing="ij")
    v = np.ones_like(grids[0])
    for g in grids:
        v = v * g
    return v.ravel()


def test_matches_bruteforce_dense():
    H = ci_matrix(300, 60, 32, seed=5, storage="f64")
    A = dense_by_loops(H)
    X = np.random.default_rng(0).standard_normal((300, 7))
    np.testing.assert_allclose(O.sym_upper_matmul(H, X), A @ X, rtol=0, atol=1e-12)
    np.testing.assert_allclose(O.sym_upper_matmul(H, X[:, 0]), A @ X[:, 0], rtol=0, atol=1e-12)


def test_laplacian_closed_form_eigenvector():
    dims = [5, 6, 7]
    H = laplacian_kron(dims)
    for ks in [(1, 1, 1), (2, 3, 1), (5, 6, 7)]:
        v = lap_eigvec(dims, ks)
        lam = sum(2 - 2 * np.cos(np.pi * k / (m + 1)) for m, k in zip(dims, ks))
        np.testing.assert_allclose(O.sym_upper_matmul(H, v), lam * v, atol=1e-12)


def test_integer_exact():
    rng = np.random.default_rng(1)
    n = 50
    rows, cols, vals = [], [], []
    for i in range(n):
        js = sorted(set([i] + list(rng.integers(i, n, size=4))))
        for j in js:
            rows.append(i); cols.append(j); vals.append(float(rng.integers(-3, 4)))
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    H = CSRUpper(n, rowptr, np.array(cols, np.int32), np.array(vals), "f64")
    X = rng.integers(-5, 6, size=(n, 3)).astype(np.float64)
    Y = O.sym_upper_matmul(H, X)
    ref = np.zeros((n, 3))
    for i, j, v in zip(rows, cols, vals):
        ref[i] += v * X[j]
        if j != i:
            ref[j] += v * X[i]
    assert np.array_equal(Y, ref)


def test_planted_mistake_is_caught():
    """A SpMM that forgets the transposed half (or double counts the diagonal) fails the pin."""
    H = ci_matrix(200, 40, 32, seed=6, storage="f64")
    A = dense_by_loops(H)
    X = np.random.default_rng(2).standard_normal((200, 3))
    U = O.to_scipy_upper(H)
    wrong1 = U @ X
    wrong2 = U @ X + U.T @ X
    assert np.abs(wrong1 - A @ X).max() > 1e-3
    assert np.abs(wrong2 - A @ X).max() > 1e-3


def test_parallel_upper_is_bitwise_the_same_product():
    """The threaded product (row ranges of U and U^T in host threads) computes every output row
    with the same sum in the same order: equal bit for bit to the single-threaded one."""
    H = ci_matrix(3001, 120, 64, seed=5, storage="f64")
    U = O.to_scipy_upper(H)
    X = np.random.default_rng(3).standard_normal((H.n, 7))
    for threads in (1, 3, 8):
        P = O.parallel_upper(H, threads)
        assert np.array_equal(O.sym_upper_matmul(H, X, P), O.sym_upper_matmul(H, X, U))
        assert np.array_equal(O.sym_upper_matmul(H, X[:, 2], P), O.sym_upper_matmul(H, X[:, 2], U))
        assert np.array_equal(P.diagonal(), U.diagonal())
