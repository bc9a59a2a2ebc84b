"""Block Lanczos, Algorithm 1 -- oracle, test infrastructure only.

V_1 = orthonormal basis of X^(0); each iteration forms W_i = (I - V V^T) H V_i
(Eq. bgs), V_{i+1} R_{i+1} = W_i (QR), appends V_{i+1} to the basis, forms
T = V^T H V (Alg. 1 "Update T_{i+1}"), solves T U = U Theta, and checks the
residual estimate of Eq. (ritzest2).

Readings:
* the basis append of Alg. 1 reads (V_i V_i); it is (V_i, V_{i+1});
* the projection of Eq. (bgs) is applied twice (CGS2) and the QR is CholQR2;
* T = V^T (H V) is formed literally from the stored H V_j blocks and symmetrised;
* the stopping test uses the exact residual norm ||W_k E_k^T q|| / |theta| (which the
  paper's ||W_k||_F ||E_k^T q|| / |theta| bounds from above); both are logged;
* "goto 16" means: skip the loop and return the current Ritz pairs.
"""
import numpy as np

from .blocks import cholqr2
from .dense import eigh_sorted
from .result import EigResult
from .spmm import sym_upper_matmul, to_scipy_upper


def _ritz(Vs, HVs, nev, passes=2):
    Vb = np.hstack(Vs)
    HVb = np.hstack(HVs)
    T = Vb.T @ HVb
    T = 0.5 * (T + T.T)
    th, Uq = eigh_sorted(T)
    W = HVs[-1].copy()
    for _ in range(passes):
        W = W - Vb @ (Vb.T @ W)
    nb = Vs[-1].shape[1]
    Ek = Uq[-nb:, :nev]                     # E_k^T q for the nev lowest
    theta = th[:nev]
    est = np.linalg.norm(W @ Ek, axis=0) / np.abs(theta)
    est_paper = np.linalg.norm(W) * np.linalg.norm(Ek, axis=0) / np.abs(theta)
    return theta, Uq[:, :nev], W, est, est_paper, Vb, HVb


def block_lanczos(H, X0, nev, tol=1e-6, maxiter=200, U=None, stop=None):
    """stop(it, theta, relres) -> True ends the iteration early (used by the hybrid)."""
    U = to_scipy_upper(H) if U is None else U
    V1, _ = cholqr2(np.asarray(X0, dtype=np.float64))
    Vs, HVs = [V1], [sym_upper_matmul(H, V1, U)]
    nb = V1.shape[1]
    hist = []
    theta, Uq, W, est, estp, Vb, HVb = _ritz(Vs, HVs, nev)
    hist.append(dict(it=0, theta=theta.copy(), relres=est.copy(), relres_paper=estp.copy()))
    conv = bool(np.all(est < tol))
    it = 0
    while not conv and it < maxiter:
        if stop is not None and stop(it, theta, est):
            break
        it += 1
        try:
            Vn, _ = cholqr2(W)
        except np.linalg.LinAlgError:
            break                                   # W rank deficient: basis exhausted
        Vs.append(Vn)
        HVs.append(sym_upper_matmul(H, Vn, U))
        theta, Uq, W, est, estp, Vb, HVb = _ritz(Vs, HVs, nev)
        hist.append(dict(it=it, theta=theta.copy(), relres=est.copy(), relres_paper=estp.copy()))
        conv = bool(np.all(est < tol))
    X = Vb @ Uq
    HX = HVb @ Uq
    nblocks = len(Vs)
    return EigResult(theta=theta, X=X, relres=est, converged=conv, iterations=it, spmm=nblocks,
                     spmv=nblocks * nb, HX=HX, history=hist)
