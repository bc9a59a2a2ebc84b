"""Pins for LOBPCG (Alg. 2) and the Jacobi preconditioner."""
import numpy as np
import scipy.sparse as sp

import oracle as O
from gen import laplacian_kron, laplacian_kron_eigs, ci_matrix, random_block, principal_submatrix, pad_rows


def test_lobpcg_laplacian_closed_form():
    dims = [11, 13, 17]
    H = laplacian_kron(dims)
    exact = laplacian_kron_eigs(dims)
    for pc in ["none", "jacobi"]:
        r = O.lobpcg(H, random_block(H.n, 8, 4), 5, tol=1e-8, precond=pc, maxiter=400)
        assert r.converged, pc
        np.testing.assert_allclose(r.theta[:5], exact[:5], rtol=1e-10)
        prev = None
        for h in r.history:
            assert np.all(h["theta"][:5] >= exact[:5] - 1e-9)
            if prev is not None:
                assert np.all(h["theta"] <= prev + 1e-9)
            prev = h["theta"]


def test_lobpcg_ci_vs_dense_and_recurrence():
    H = ci_matrix(2000, 100, 64, seed=1, storage="f64")
    lam, _ = O.lowest_eigpairs(O.to_dense(H), 5)
    Z0 = O.lowest_eigpairs(O.to_dense(principal_submatrix(H, 200)), 8)[1]
    r = O.lobpcg(H, pad_rows(Z0, H.n), 5, tol=1e-8)
    assert r.converged
    np.testing.assert_allclose(r.theta[:5], lam, rtol=1e-10)
    # H X carried by the recurrences (Eqs. upd1-upd2) equals H applied to X
    np.testing.assert_allclose(r.HX, O.sym_upper_matmul(H, r.X), atol=1e-9)
    np.testing.assert_allclose(r.X.T @ r.X, np.eye(8), atol=1e-10)


def test_jacobi_precond_floor():
    d = np.array([0.0, 1.0, 5.0])
    R = np.ones((3, 2))
    W = O.jacobi_apply(d, np.array([0.95, 2.0]), R, floor=0.1)
    # (0-0.95) -> -0.95; (1-0.95) = 0.05 -> floored to 0.1; (5-0.95) = 4.05
    np.testing.assert_allclose(W[:, 0], [1 / -0.95, 1 / 0.1, 1 / 4.05])
    np.testing.assert_allclose(W[:, 1], [1 / -2.0, 1 / -1.0, 1 / 3.0])


def test_lobpcg_and_lanczos_match_eigsh_at_20000():
    """The plain FP64 workload (n = 20,000, ~100 nnz/row, block pattern 64, n_ev = 5, block 8):
    the oracle's LOBPCG and Lanczos against scipy's ARPACK (eigsh, smallest algebraic)."""
    import scipy.sparse.linalg as sla
    H = ci_matrix(20000, 100, 64, seed=1, storage="f64")
    U = O.to_scipy_upper(H)
    A = (U + U.T - sp.diags(U.diagonal())).tocsr()
    ref = np.sort(sla.eigsh(A, k=5, which="SA", tol=1e-12)[0])
    r = O.lobpcg(H, random_block(H.n, 8, 3), 5, tol=1e-8, maxiter=500, U=U)
    assert r.converged
    np.testing.assert_allclose(np.sort(r.theta[:5]), ref, rtol=1e-9, atol=1e-12)
    lz = O.lanczos(H, np.random.default_rng(4).standard_normal(H.n), 5, tol=1e-8)
    np.testing.assert_allclose(np.sort(lz.theta[:5]), ref, rtol=1e-9, atol=1e-12)
