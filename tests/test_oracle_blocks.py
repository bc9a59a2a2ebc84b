"""Pins for Gram, CholQR2 and Rayleigh-Ritz (Alg. 2-3, Eq. rreig)."""
import numpy as np
import pytest

import oracle as O
from gen import laplacian_kron, laplacian_kron_eigs


def test_cholqr2_orthonormal_and_factor():
    X = np.random.default_rng(0).standard_normal((500, 12))
    Q, R = O.cholqr2(X)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-13)
    np.testing.assert_allclose(Q @ R, X, atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0)


def test_cholqr2_ill_conditioned():
    t = np.linspace(0.1, 1.0, 2000)
    X = np.stack([t ** j for j in range(8)], axis=1)      # Vandermonde, cond ~ 1e6
    assert np.linalg.cond(X) > 1e4
    Q, R = O.cholqr2(X)
    assert np.abs(Q.T @ Q - np.eye(8)).max() < 1e-11
    np.testing.assert_allclose(Q @ R, X, atol=1e-10)


def test_cholqr_breaks_on_rank_deficient():
    X = np.random.default_rng(1).standard_normal((100, 3))
    X = np.hstack([X, X[:, :1]])
    with pytest.raises(np.linalg.LinAlgError):
        O.cholqr(X)


def test_rayleigh_ritz_exact_invariant_subspace():
    dims = [4, 5, 6]
    H = laplacian_kron(dims)
    lam, V = O.lowest_eigpairs(O.to_dense(H), 6)
    M = np.random.default_rng(3).standard_normal((6, 6))
    S = V @ M                                             # same span, not orthonormal
    HS = O.sym_upper_matmul(H, S)
    theta, C = O.rayleigh_ritz(S, HS, 4)
    np.testing.assert_allclose(theta, laplacian_kron_eigs(dims)[:4], atol=1e-12)
    np.testing.assert_allclose(C.T @ (S.T @ S) @ C, np.eye(4), atol=1e-12)


def test_rayleigh_ritz_full_space_is_dense_solve():
    dims = [3, 3, 4]
    H = laplacian_kron(dims)
    S = np.random.default_rng(4).standard_normal((36, 36))
    theta, C = O.rayleigh_ritz(S, O.sym_upper_matmul(H, S), 5)
    np.testing.assert_allclose(theta, laplacian_kron_eigs(dims)[:5], atol=1e-10)


def test_gram():
    A = np.arange(12.0).reshape(4, 3)
    np.testing.assert_array_equal(O.gram(A), A.T @ A)
    assert O.gram(A)[0, 0] == 0 + 9 + 36 + 81
