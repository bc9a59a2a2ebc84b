"""Chebyshev-filtered subspace iteration, Algorithm 3 -- oracle, test infrastructure only.

Filter: T_m((H - cI)/e) applied by the three-term recurrence of Eq. (chebypoly),
c = (lambda_ub + lambda_F)/2, e = (lambda_ub - lambda_F)/2; then CholeskyQR, the
Rayleigh-Ritz step T = Q^T H Q, T S = S Theta, Q <- Q S, and the relative residual
test on R = H Q - Q Theta.  lambda_ub follows Sec. 3.2: ten Lanczos steps, the
largest Ritz pair (theta_10, u_10), lambda_ub = theta_10 + ||r_10||.  Converged
vectors are locked (Sec. 3.2): H is not applied to them, but they stay in the
Rayleigh-Ritz step.

Readings:
* first filter step W = (HQ - cQ)/e, i.e. T_1(t) = t of Eq. (chebypoly) (the listing's
  factor 2 would make the filter a second-kind polynomial U_d);
* "CholeskyQR(H, X^(0))" is CholQR2(X^(0)); before CholQR2 the filtered columns are
  scaled to unit norm (span unchanged);
* lambda_F: the synthetic spectrum is not negative, so lambda_F = 0 (the paper's value
  for bound states) would filter nothing; lambda_F is the largest Ritz value of the
  current block, starting from a Rayleigh-Ritz step on the orthonormalised X^(0);
* H Q after CholQR2 is obtained as (H Y) R^{-1}, where H Y is the filter's last product
  for unlocked columns and H Q_old for locked ones; each iteration therefore costs d
  products with the active columns;
* ||r_10|| uses the Lanczos relation ||H u - theta u|| = beta_10 |e_10^T q|.
"""
import numpy as np
import scipy.linalg as sla

from .blocks import cholqr2, rayleigh_ritz
from .dense import eigh_sorted
from .result import EigResult
from .spmm import sym_upper_matmul, to_scipy_upper


def lambda_ub_estimate(H, v, steps=10, U=None):
    U = to_scipy_upper(H) if U is None else U
    v = np.asarray(v, dtype=np.float64).ravel()
    v = v / np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    for j in range(steps):
        w = sym_upper_matmul(H, V[-1], U)
        alpha.append(float(V[-1] @ w))
        Vm = np.array(V).T
        for _ in range(2):
            w = w - Vm @ (Vm.T @ w)
        b = float(np.linalg.norm(w))
        beta.append(b)
        if b == 0.0:
            break
        V.append(w / b)
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:k - 1], 1) + np.diag(beta[:k - 1], -1)
    th, Q = eigh_sorted(T)
    return float(th[-1] + beta[k - 1] * abs(Q[-1, -1])), k


def cheb_step(HW, W, Qp, c, e):
    """One step of the three-term recurrence of Eq. (chebypoly) on (H - cI)/e:
    T_{j}(t) = 2 t T_{j-1}(t) - T_{j-2}(t), i.e. Y = 2 (H W - c W) / e - Q_prev."""
    return 2.0 * (HW - c * W) / e - Qp


def cheb_filter(H, Q, HQ, deg, c, e, active=None, U=None):
    """Y = T_deg((H - cI)/e) Q on the active columns (others returned unchanged) and
    H Y for the active columns' last recurrence input.  Returns (Y, products)."""
    U = to_scipy_upper(H) if U is None else U
    nb = Q.shape[1]
    act = np.ones(nb, bool) if active is None else np.asarray(active, bool)
    Qa, HQa = Q[:, act], HQ[:, act]
    W = (HQa - c * Qa) / e
    Qp = Qa
    products = 0
    for _ in range(2, deg + 1):
        HW = sym_upper_matmul(H, W, U)
        products += 1
        Y = cheb_step(HW, W, Qp, c, e)
        Qp, W = W, Y
    Y = Q.copy()
    Y[:, act] = W
    return Y, products


def chebfsi(H, X0, nev, deg=10, tol=1e-6, maxiter=100, lambda_ub=None, v_ub=None, U=None):
    U = to_scipy_upper(H) if U is None else U
    X0 = np.asarray(X0, dtype=np.float64)
    nb = X0.shape[1]
    spmv = 0
    if lambda_ub is None:
        lambda_ub, k = lambda_ub_estimate(H, v_ub, 10, U)
        spmv += k
    Q, _ = cholqr2(X0)
    HQ = sym_upper_matmul(H, Q, U)
    spmv += nb
    theta, S = rayleigh_ritz(Q, HQ, nb)
    Q, HQ = Q @ S, HQ @ S
    R = HQ - Q * theta[None, :]
    relres = np.linalg.norm(R, axis=0) / np.abs(theta)
    lam_f = float(theta[-1])
    hist = [dict(it=0, theta=theta.copy(), relres=relres.copy(), lambda_f=lam_f)]
    conv = bool(np.all(relres[:nev] < tol))
    it = 0
    while not conv and it < maxiter:
        it += 1
        locked = relres < tol
        act = ~locked
        c, e = 0.5 * (lambda_ub + lam_f), 0.5 * (lambda_ub - lam_f)
        Y, prods = cheb_filter(H, Q, HQ, deg, c, e, act, U)
        spmv += prods * int(act.sum())
        HY = HQ.copy()
        HY[:, act] = sym_upper_matmul(H, Y[:, act], U)
        spmv += int(act.sum())
        s = np.linalg.norm(Y, axis=0)
        Y, HY = Y / s[None, :], HY / s[None, :]
        Q, Rq = cholqr2(Y)
        HQ = sla.solve_triangular(Rq, HY.T, trans="T", lower=False).T
        T = Q.T @ HQ
        theta, Sv = eigh_sorted(0.5 * (T + T.T))
        Q, HQ = Q @ Sv, HQ @ Sv
        R = HQ - Q * theta[None, :]
        relres = np.linalg.norm(R, axis=0) / np.abs(theta)
        lam_f = float(theta[-1])
        hist.append(dict(it=it, theta=theta.copy(), relres=relres.copy(), lambda_f=lam_f,
                         active=int(act.sum())))
        conv = bool(np.all(relres[:nev] < tol))
    return EigResult(theta=theta[:nev], X=Q[:, :nev], relres=relres[:nev], converged=conv,
                     iterations=it, spmm=None, spmv=spmv, HX=HQ[:, :nev], history=hist,
                     extra=dict(lambda_ub=lambda_ub, theta_all=theta, X_all=Q))
