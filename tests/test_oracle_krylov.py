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


def test_block_lanczos_thick_restart_closed_form_and_bounded_basis():
    """Restarted after 4 blocks of 8 (Sec. 2.2), keeping 16 Ritz vectors: the same lowest
    eigenvalues as the closed form, the exact residual estimate, a basis that never exceeds the
    restart size, and Ritz values that still never fall below the eigenvalues (the basis stays a
    subspace: Rayleigh-Ritz values bound the eigenvalues from above)."""
    H = laplacian_kron(DIMS)
    exact = laplacian_kron_eigs(DIMS)
    r = O.block_lanczos(H, random_block(H.n, 8, 2), 5, tol=1e-8, maxiter=400, restart=4, keep=16)
    assert r.converged and r.extra["restarts"] >= 2
    np.testing.assert_allclose(r.theta, exact[:5], rtol=1e-10)
    assert max(h["basis"] for h in r.history) <= 4 * 8
    for h in r.history:
        assert np.all(h["theta"][:5] >= exact[:5] - 1e-9)
    tr = O.true_relres(H, r.theta, r.X)
    np.testing.assert_allclose(tr, r.relres, rtol=1e-5, atol=1e-12)


def test_thick_restart_keeps_the_krylov_schur_form():
    """Right after a restart the basis [Y, V_new] satisfies H Y = Y Theta + V_new S: the kept block
    of T = V^T H V is diag(theta_1..p), and H Y has no component outside span(Y, V_new)."""
    H = ci_matrix(600, 40, 32, seed=3, storage="f64")
    U = O.to_scipy_upper(H)
    nb, p = 4, 6
    V1, _ = O.cholqr2(random_block(H.n, nb, 5))
    Vs, HVs = [V1], [O.sym_upper_matmul(H, V1, U)]
    for _ in range(4):                                       # a Krylov basis of five blocks
        Vb, HVb = np.hstack(Vs), np.hstack(HVs)
        W = HVs[-1] - Vb @ (Vb.T @ HVs[-1])
        W = W - Vb @ (Vb.T @ W)
        Vn, _ = O.cholqr2(W)
        Vs.append(Vn); HVs.append(O.sym_upper_matmul(H, Vn, U))
    Vb, HVb = np.hstack(Vs), np.hstack(HVs)
    T = Vb.T @ HVb
    th, Uq = np.linalg.eigh(0.5 * (T + T.T))
    W = HVs[-1] - Vb @ (Vb.T @ HVs[-1])
    W = W - Vb @ (Vb.T @ W)
    (Y, Vn), (HY, _) = O.thick_restart(Vb, HVb, Uq, p, W)
    np.testing.assert_allclose(HY, O.sym_upper_matmul(H, Y, U), atol=1e-10)   # linearity
    B = np.hstack([Y, Vn])
    np.testing.assert_allclose(B.T @ B, np.eye(p + nb), atol=1e-12)
    np.testing.assert_allclose(Y.T @ HY, np.diag(th[:p]), atol=1e-10)
    out = HY - B @ (B.T @ HY)
    assert np.linalg.norm(out) < 1e-9 * np.linalg.norm(HY)


def test_thick_restart_keeping_the_wrong_end_is_caught():
    """A planted mistake -- keeping the highest Ritz vectors -- leaves the lowest pairs unconverged
    or wrong, which the closed form rejects."""
    H = laplacian_kron(DIMS)
    exact = laplacian_kron_eigs(DIMS)
    bl = __import__("importlib").import_module("oracle.block_lanczos")
    good = bl.thick_restart

    def wrong(Vb, HVb, Uq, p, W):
        return good(Vb, HVb, Uq[:, ::-1], p, W)
    bl.thick_restart = wrong
    try:
        r = O.block_lanczos(H, random_block(H.n, 8, 2), 5, tol=1e-8, maxiter=60, restart=4, keep=16)
    finally:
        bl.thick_restart = good
    assert not (r.converged and np.allclose(r.theta, exact[:5], rtol=1e-10))
