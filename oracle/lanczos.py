"""Lanczos with full orthogonalisation (Sec. 2.1) -- oracle, test infrastructure only.

Builds the Krylov basis of Eq. (krylov) by the Gram-Schmidt step of Eq. (gs),
w_j = (I - V_j V_j^T) H v_j, v_{j+1} = w_j / ||w_j||, the tridiagonal T_k of
Eq. (lanfac) (alpha_j = v_j^T H v_j, beta_j = ||w_j||), the Ritz pairs of Eq. (trideig),
and the residual estimate of Eq. (ritzest1): ||w_k|| |e_k^T q| / |theta|.

Reading: the projection of Eq. (gs) is applied twice (classical Gram-Schmidt with
one re-orthogonalisation) -- identical in exact arithmetic, and what "full
orthogonalisation" needs in floating point.
"""
import numpy as np

from .dense import eigh_sorted
from .result import EigResult
from .spmm import sym_upper_matmul, to_scipy_upper


def lanczos(H, v0, nev, tol=1e-6, maxiter=1000, U=None, passes=2):
    U = to_scipy_upper(H) if U is None else U
    v = np.asarray(v0, dtype=np.float64).ravel()
    v = v / np.linalg.norm(v)
    n = v.size
    V = np.zeros((n, min(maxiter, n) + 1))
    V[:, 0] = v
    alpha, beta, hist = [], [], []
    theta = X = est = None
    conv = False
    j = 0
    for j in range(1, min(maxiter, n) + 1):
        w = sym_upper_matmul(H, V[:, j - 1], U)
        alpha.append(float(V[:, j - 1] @ w))
        for _ in range(passes):
            w = w - V[:, :j] @ (V[:, :j].T @ w)
        b = float(np.linalg.norm(w))
        beta.append(b)
        T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
        th, Q = eigh_sorted(T)
        k = min(nev, j)
        theta = th[:k]
        est = b * np.abs(Q[-1, :k]) / np.abs(theta)
        hist.append(dict(it=j, theta=theta.copy(), relres=est.copy()))
        if k == nev and np.all(est < tol):
            conv = True
            X = V[:, :j] @ Q[:, :k]
            break
        if b <= 1e-14 * max(1.0, np.max(np.abs(th))):
            conv = k == nev
            X = V[:, :j] @ Q[:, :k]
            break
        V[:, j] = w / b
    if X is None:
        X = V[:, :j] @ Q[:, :min(nev, j)]
    return EigResult(theta=theta, X=X, relres=est, converged=conv, iterations=j, spmm=j, spmv=j,
                     history=hist, extra=dict(T_alpha=np.array(alpha), T_beta=np.array(beta)))
