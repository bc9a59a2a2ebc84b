"""Pins for Lanczos (Sec. 2.1) and block Lanczos (Alg. 1)."""
import numpy as np

import oracle as O
from gen import laplacian_kron, laplacian_kron_eigs, ci_matrix, random_block

DIMS = [11, 13, 17]          # non-commensurate: simple lowest eigenvalues


def _check_monotone(hist, exact):
    prev = None
    for h in hist:
        th = h["theta"]
        k = min(len(th), len(exact))
        assert np.all(th[:k] >= exact[:k] - 1e-9)                 # Cauchy interlacing
        if prev is not None:
            m = min(len(prev), k)
            assert np.all(th[:m] <= prev[:m] + 1e-9)              # nested subspaces
        prev = th


def test_lanczos_laplacian_closed_form():
    H = laplacian_kron(DIMS)
    exact = laplacian_kron_eigs(DIMS)
    v0 = random_block(H.n, 1, 1)[:, 0]
    r = O.lanczos(H, v0, 5, tol=1e-8)
    assert r.converged
    np.testing.assert_allclose(r.theta, exact[:5], rtol=1e-10)
    assert np.all(O.true_relres(H, r.theta, r.X) < 1e-6)
    _check_monotone(r.history, exact)


def test_lanczos_tridiagonal_recurrence():
    """On T_m from e_1 the Lanczos coefficients are exactly alpha = 2, beta = 1."""
    m = 12
    H = laplacian_kron([m])
    e1 = np.zeros(m); e1[0] = 1
    r = O.lanczos(H, e1, 3, tol=0.0, maxiter=m)
    a, b = r.extra["T_alpha"], r.extra["T_beta"]
    np.testing.assert_allclose(a, 2.0, atol=1e-13)
    np.testing.assert_allclose(b[:-1], 1.0, atol=1e-13)
    assert b[-1] < 1e-12                                        # invariant subspace reached


def test_block_lanczos_laplacian_closed_form():
    H = laplacian_kron(DIMS)
    exact = laplacian_kron_eigs(DIMS)
    X0 = random_block(H.n, 8, 2)
    r = O.block_lanczos(H, X0, 5, tol=1e-8)
    assert r.converged
    np.testing.assert_allclose(r.theta, exact[:5], rtol=1e-10)
    _check_monotone(r.history, exact)
    # the exact estimate equals the true residual norm
    tr = O.true_relres(H, r.theta, r.X)
    np.testing.assert_allclose(tr, r.relres, rtol=1e-5, atol=1e-12)
    for h in r.history:
        assert np.all(h["relres_paper"] >= h["relres"] * (1 - 1e-12))  # paper's bound is an upper bound


def test_block_lanczos_ci_vs_dense():
    H = ci_matrix(1500, 80, 64, seed=2, storage="f64")
    lam, _ = O.lowest_eigpairs(O.to_dense(H), 5)
    r = O.block_lanczos(H, random_block(H.n, 8, 3), 5, tol=1e-7)
    assert r.converged
    np.testing.assert_allclose(r.theta, lam, rtol=1e-9)
