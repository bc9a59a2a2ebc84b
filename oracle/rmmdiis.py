"""RMM-DIIS, Algorithm 4, batched over eigenvectors (Sec. 4.2) -- oracle, test
infrastructure only.

Per eigenvector j: normalise x^(0), theta^(0) = <x, Hx>, r^(0) = Hx - theta x; the
first iteration uses x~ = x^(0), r~ = r^(0).  Iteration l > 1 solves the constrained
least-squares problem of Eqs. (xsum)-(rmm) over the last s residuals, forms x~
(Eq. xsum), normalises it, and sets r~ = H x~ - theta~ x~ with
theta~ = <x~, H x~> / <x~, x~>.  Then the 2x2 Rayleigh-Ritz problem of Eq. (rr) on
W = (x~, r~) gives x^(l) = W g (Eq. xuwg) with g the eigenvector of the smaller
eigenvalue, and r^(l) = H x^(l) - theta^(l) x^(l); stop when ||r|| / |theta| < tol.
All eigenvectors advance in lock-step (the batched SpMM of Sec. 4.3); converged
ones are no longer updated.

Readings:
* sum limits (garbled as min{0, l-s} / min{l-s}): i runs over the last
  s = min(l, s_max) iterates, i in [l - s, l - 1];
* the listing's "r~ = sum alpha x" is a typo; the text's r~ = H x~ - theta~ x~ is used;
* the constrained problem is solved by the substitution alpha_{l-1} = 1 - sum of the
  others (text after Eq. rmm), i.e. an unconstrained least-squares problem in the
  differences r^(i) - r^(l-1), solved with numpy.linalg.lstsq;
* x^(l) is normalised so that ||x^(l)|| = 1 (g^T (W^T W) g = 1), and the sign of g -- which the
  paper leaves open, and which the affine DIIS constraint of Eq. (alphasum) is not invariant to --
  is fixed as g_1 <= 0, the sign LAPACK's generalized symmetric eigensolver returns for these 2x2
  pencils (so consecutive iterates alternate in sign, as in a MATLAB implementation built on eig);
  with g_1 >= 0 instead the iteration stagnates on interior pairs of the CI-shaped test matrices;
* optional preconditioned variant (precond="jacobi"): the 2x2 subspace is
  W = (x~, K^{-1} r~) with the Jacobi K^{-1} of oracle.precond at theta~; the plain
  method of Alg. 4 is precond="none" (the default);
* SpMV count as in Sec. 2.6: one per eigenvector per iteration (the product H r~; H x~
  and H x follow by linearity in an implementation) plus the initial H x^(0) unless
  the caller supplies it.
"""
import numpy as np
import scipy.linalg as sla

from .precond import jacobi_apply
from .result import EigResult
from .spmm import sym_upper_matmul, to_scipy_upper


def diis_coefficients(rs):
    """alpha minimising ||sum_i alpha_i r_i|| subject to sum_i alpha_i = 1 (Eqs. alphasum,
    rmm), by substituting alpha_last = 1 - sum_{i<last} alpha_i.  rs: list, oldest first."""
    s = len(rs)
    if s == 1:
        return np.ones(1)
    rl = np.asarray(rs[-1], dtype=np.float64)
    D = np.stack([np.asarray(r, dtype=np.float64) - rl for r in rs[:-1]], axis=1)
    a, *_ = np.linalg.lstsq(D, -rl, rcond=None)
    return np.concatenate([a, [1.0 - a.sum()]])


def diis_extrapolate(xs, rs, s_max):
    """x~ of Eq. (xsum) for one eigenvector, normalised: the DIIS combination (Eqs. alphasum,
    rmm) of the newest s = min(len(xs), s_max) iterates, i in [l - s, l - 1] (the reading of the
    garbled sum limits).  xs, rs: iterate and residual histories, oldest first."""
    s = min(len(xs), s_max)
    alpha = diis_coefficients(rs[-s:])
    xt = sum(al * np.asarray(xv, dtype=np.float64) for al, xv in zip(alpha, xs[-s:]))
    return xt / np.linalg.norm(xt)


def rr2(x, r, Hx, Hr):
    """Smaller eigenpair of the 2x2 pencil (W^T H W, W^T W), W = (x, r) (Eq. rr).
    Returns (theta, g) with g^T (W^T W) g = 1 and g_1 <= 0.  Falls back to the Rayleigh quotient of x
    when W^T W is numerically singular."""
    A = np.array([[x @ Hx, x @ Hr], [r @ Hx, r @ Hr]], dtype=np.float64)
    A = 0.5 * (A + A.T)
    B = np.array([[x @ x, x @ r], [r @ x, r @ r]], dtype=np.float64)
    B = 0.5 * (B + B.T)
    try:
        w, G = sla.eigh(A, B)
        g = G[:, 0]
        return float(w[0]), (-g if g[0] > 0 else g)
    except np.linalg.LinAlgError:
        nx = np.sqrt(B[0, 0])
        return float(A[0, 0] / B[0, 0]), np.array([1.0 / nx, 0.0])


def rmmdiis(H, X0, tol=1e-6, maxiter=200, s_max=10, HX0=None, U=None, precond="none", floor=2.0):
    U = to_scipy_upper(H) if U is None else U
    diagH = U.diagonal()
    X0 = np.asarray(X0, dtype=np.float64)
    n, nev = X0.shape
    nrm = np.linalg.norm(X0, axis=0)
    X = X0 / nrm[None, :]
    spmv = 0
    if HX0 is None:
        HX = sym_upper_matmul(H, X, U)
        spmv += nev
    else:
        HX = np.asarray(HX0, dtype=np.float64) / nrm[None, :]
    theta = np.einsum("ij,ij->j", X, HX)
    R = HX - X * theta[None, :]
    xh = [[X[:, j].copy()] for j in range(nev)]
    rh = [[R[:, j].copy()] for j in range(nev)]
    relres = np.linalg.norm(R, axis=0) / np.abs(theta)
    done = relres < tol
    iters = np.zeros(nev, dtype=int)
    hist = [dict(it=0, theta=theta.copy(), relres=relres.copy())]
    spmm = 0
    it = 0
    while not np.all(done) and it < maxiter:
        it += 1
        act = np.nonzero(~done)[0]
        Xt = np.zeros((n, act.size))
        for a, j in enumerate(act):
            if it == 1:
                Xt[:, a] = X[:, j]
            else:
                Xt[:, a] = diis_extrapolate(xh[j], rh[j], s_max)
        HXt = sym_upper_matmul(H, Xt, U)
        tht = np.einsum("ij,ij->j", Xt, HXt) / np.einsum("ij,ij->j", Xt, Xt)
        Rt = HXt - Xt * tht[None, :]
        if precond == "jacobi":
            Rt = jacobi_apply(diagH, tht, Rt, floor)
        HRt = sym_upper_matmul(H, Rt, U)
        spmm += 1
        spmv += act.size
        Xn = np.zeros_like(Xt)
        thn = np.zeros(act.size)
        for a in range(act.size):
            thn[a], g = rr2(Xt[:, a], Rt[:, a], HXt[:, a], HRt[:, a])
            Xn[:, a] = g[0] * Xt[:, a] + g[1] * Rt[:, a]
            Xn[:, a] /= np.linalg.norm(Xn[:, a])
        HXn = sym_upper_matmul(H, Xn, U)
        for a, j in enumerate(act):
            th = float(Xn[:, a] @ HXn[:, a])
            r = HXn[:, a] - th * Xn[:, a]
            X[:, j], HX[:, j], theta[j] = Xn[:, a], HXn[:, a], th
            xh[j].append(Xn[:, a].copy())
            rh[j].append(r)
            relres[j] = np.linalg.norm(r) / abs(th)
            iters[j] += 1
            if relres[j] < tol:
                done[j] = True
        hist.append(dict(it=it, theta=theta.copy(), relres=relres.copy()))
    return EigResult(theta=theta, X=X, relres=relres, converged=bool(np.all(done)), iterations=it,
                     spmm=spmm, spmv=spmv, HX=HX, history=hist, extra=dict(per_vector_iterations=iters))
