"""LOBPCG, Algorithm 2 -- oracle, test infrastructure only.

Initial Rayleigh-Ritz on X^(0); then per iteration W = K^{-1} R (Eq. wblock),
S = [X W P] (Eq. rrsubspace), Rayleigh-Ritz on the pencil (S^T H S, S^T S)
(Eq. rreig), X <- S C (Eq. xupd), P <- W C_2 + P C_3 (Eq. pupd), and H X, H P by the
recurrences of Eqs. (upd1)-(upd2), so the only product with H is H W.  Convergence:
relative residual norms ||R_j|| / |theta_j| of the leading n_ev columns.

Readings:
* P^(0) is empty, so S = [X W] in the first iteration;
* K^{-1} is the Jacobi preconditioner of oracle.precond (precond="none" gives K = I);
* the Rayleigh-Ritz step works on the numerically independent part of span(S)
  (oracle.blocks.rayleigh_ritz_projected), which is the exact pencil solution whenever
  S^T S is nonsingular;
* the recurrences of Eqs. (upd1)-(upd2) are exact in exact arithmetic but carry rounding: once
  the Rayleigh-Ritz coefficients on unit-norm basis columns exceed 1e3 (a nearly dependent S,
  Sec. 2.3's ill-conditioned pencil), or every 20 iterations, H X and H P are recomputed by
  their definition (products not counted in `spmm`, which counts the method's own products).
  Without this the Ritz values of long runs drifted below the spectrum (to -1e76 on a
  20,000-row CI matrix from a random start).
"""
import numpy as np

from .blocks import rayleigh_ritz
from .precond import jacobi_apply
from .result import EigResult
from .spmm import sym_upper_matmul, to_scipy_upper


def lobpcg(H, X0, nev, tol=1e-6, maxiter=500, precond="jacobi", floor=2.0, U=None, stop=None,
           diagH=None):
    """stop(it, theta, relres) -> True ends the iteration early (used by the hybrid)."""
    U = to_scipy_upper(H) if U is None else U
    X0 = np.asarray(X0, dtype=np.float64)
    nb = X0.shape[1]
    if diagH is None:
        diagH = U.diagonal()
    HX0 = sym_upper_matmul(H, X0, U)
    spmm = 1
    theta, C = rayleigh_ritz(X0, HX0, nb)
    X, HX = X0 @ C, HX0 @ C
    R = HX - X * theta[None, :]
    P = HP = None
    relres = np.linalg.norm(R, axis=0) / np.abs(theta)
    hist = [dict(it=0, theta=theta.copy(), relres=relres.copy())]
    conv = bool(np.all(relres[:nev] < tol))
    it = 0
    since = 0
    refreshed = 0
    while not conv and it < maxiter:
        if stop is not None and stop(it, theta, relres):
            break
        it += 1
        W = jacobi_apply(diagH, theta, R, floor) if precond == "jacobi" else R.copy()
        HW = sym_upper_matmul(H, W, U)
        spmm += 1
        if P is None:
            S, HS = np.hstack([X, W]), np.hstack([HX, HW])
        else:
            S, HS = np.hstack([X, W, P]), np.hstack([HX, HW, HP])
        theta, C = rayleigh_ritz(S, HS, nb)
        C2 = C[nb:2 * nb]
        Pn = W @ C2
        HPn = HW @ C2
        if P is not None:
            C3 = C[2 * nb:]
            Pn = Pn + P @ C3
            HPn = HPn + HP @ C3
        X, HX = S @ C, HS @ C
        P, HP = Pn, HPn
        since += 1
        cmax = np.max(np.abs(C) * np.linalg.norm(S, axis=0)[:, None])
        if cmax > 1e3 or since >= 20:
            HX = sym_upper_matmul(H, X, U)
            HP = sym_upper_matmul(H, P, U)
            since = 0
            refreshed += 1
        R = HX - X * theta[None, :]
        relres = np.linalg.norm(R, axis=0) / np.abs(theta)
        hist.append(dict(it=it, theta=theta.copy(), relres=relres.copy()))
        conv = bool(np.all(relres[:nev] < tol))
    return EigResult(theta=theta, X=X, relres=relres, converged=conv, iterations=it, spmm=spmm,
                     spmv=spmm * nb, HX=HX, history=hist, extra=dict(refreshed=refreshed))
