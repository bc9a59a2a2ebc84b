"""LOBPCG, Algorithm 2 -- oracle, test infrastructure only.

Initial Rayleigh-Ritz on X^(0); then per iteration W = K^{-1} R (Eq. wblock),
S = [X W P] (Eq. rrsubspace), Rayleigh-Ritz on the pencil (S^T H S, S^T S)
(Eq. rreig), X <- S C (Eq. xupd), P <- W C_2 + P C_3 (Eq. pupd); the method's only product
with H is H W (H X and H P follow from Eqs. (upd1)-(upd2)).  Convergence: relative residual
norms ||R_j|| / |theta_j| of the leading n_ev columns.

Readings:
* P^(0) is empty, so S = [X W] in the first iteration;
* K^{-1} is the Jacobi preconditioner of oracle.precond (precond="none" gives K = I);
* the Rayleigh-Ritz step works on the numerically independent part of span(S)
  (oracle.blocks.rayleigh_ritz_projected), which is the exact pencil solution whenever
  S^T S is nonsingular;
* H X and H P: Eqs. (upd1)-(upd2) update them by recurrences, which are exact in exact
  arithmetic; the oracle needs no speed, so it forms both by their definition (H times the
  updated block) every iteration instead, and counts in `spmm` only the method's own product
  H W.  This keeps the oracle free of any rule for when rounding in the recurrences has grown
  too large (a recurrence run on a nearly dependent S drifts: its Ritz values fell below the
  spectrum on long runs).
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
        P = W @ C[nb:2 * nb]
        if S.shape[1] > 2 * nb:
            P = P + S[:, 2 * nb:] @ C[2 * nb:]
        X = S @ C
        # H X and H P by definition (exact counterparts of Eqs. upd1-upd2; not counted)
        HX = sym_upper_matmul(H, X, U)
        HP = sym_upper_matmul(H, P, U)
        R = HX - X * theta[None, :]
        relres = np.linalg.norm(R, axis=0) / np.abs(theta)
        hist.append(dict(it=it, theta=theta.copy(), relres=relres.copy()))
        conv = bool(np.all(relres[:nev] < tol))
    return EigResult(theta=theta, X=X, relres=relres, converged=conv, iterations=it, spmm=spmm,
                     spmv=spmm * nb, HX=HX, history=hist)
