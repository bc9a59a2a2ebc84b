"""Tall-skinny dense block operations (oracle; test infrastructure only).

* gram: A^T B, the "level 3 BLAS" products of Sec. 1 used by the Rayleigh-Ritz
  procedure (Eq. rreig) and by block Gram-Schmidt (Eq. bgs).
* cholqr / cholqr2: the CholeskyQR orthonormalisation named in Alg. 3 (line 3 and
  line 10): G = X^T X = R^T R, Q = X R^{-1}; CholQR2 applies it twice.
* rayleigh_ritz: the Rayleigh-Ritz procedure of Sec. 2.3 -- the n_b leftmost
  eigenpairs of the pencil (S^T H S, S^T S) (Eq. rreig), C normalised so that
  C^T (S^T S) C = I.
"""
import numpy as np
import scipy.linalg as sla

from .dense import eigh_sorted


def gram(A, B=None):
    A = np.asarray(A, dtype=np.float64)
    B = A if B is None else np.asarray(B, dtype=np.float64)
    return A.T @ B


BREAKDOWN_RTOL = 1e-14


def cholqr(X):
    """One CholeskyQR pass.  Returns (Q, R) with X = Q R, R upper triangular.
    Raises numpy.linalg.LinAlgError when X^T X is not numerically positive definite:
    a Cholesky failure, or a squared pivot below BREAKDOWN_RTOL * max diag(X^T X)."""
    X = np.asarray(X, dtype=np.float64)
    G = X.T @ X
    L = np.linalg.cholesky(0.5 * (G + G.T))
    if np.min(np.diag(L)) ** 2 <= BREAKDOWN_RTOL * np.max(np.diag(G)):
        raise np.linalg.LinAlgError("CholeskyQR breakdown: numerically rank-deficient block")
    R = L.T
    Q = sla.solve_triangular(R, X.T, trans="T", lower=False).T
    return Q, R


def cholqr2(X):
    """CholeskyQR applied twice (X = Q1 R1, Q1 = Q R2, R = R2 R1)."""
    Q1, R1 = cholqr(X)
    Q, R2 = cholqr(Q1)
    return Q, R2 @ R1


def orthonormal_basis(G, drop_tol=1e-12):
    """Coefficients Q (k x m) with Q^T G Q = I spanning the numerically nonsingular part
    of the Gram matrix G = S^T S.  Columns are first scaled to unit norm (the span is
    unchanged); eigen-directions of the scaled Gram below drop_tol * max are dropped."""
    d = np.sqrt(np.maximum(np.diag(G), 1e-300))
    Dinv = 1.0 / d
    Gs = G * Dinv[:, None] * Dinv[None, :]
    w, V = eigh_sorted(Gs)
    keep = w > drop_tol * w[-1]
    Q = (V[:, keep] / np.sqrt(w[keep])[None, :]) * Dinv[:, None]
    return Q


def rayleigh_ritz_projected(A, G, nb, drop_tol=1e-12):
    """Leftmost nb eigenpairs of the projected pencil (A, G) = (S^T H S, S^T S)
    (Eq. rreig).  Returns (theta[nb], C[k, nb]) with C^T G C = I."""
    A = 0.5 * (A + A.T)
    G = 0.5 * (G + G.T)
    Q = orthonormal_basis(G, drop_tol)
    T = Q.T @ A @ Q
    w, Z = eigh_sorted(T)
    m = min(nb, w.size)
    return w[:m].copy(), Q @ Z[:, :m]


def rayleigh_ritz(S, HS, nb, drop_tol=1e-12):
    """Rayleigh-Ritz on span(S) given HS = H S: returns (theta, C) of Eq. (rreig)."""
    S = np.asarray(S, dtype=np.float64)
    HS = np.asarray(HS, dtype=np.float64)
    return rayleigh_ritz_projected(S.T @ HS, S.T @ S, nb, drop_tol)
