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
* "goto 16" means: skip the loop and return the current Ritz pairs;
* restart (Sec. 2.2: "restart the algorithm after d iterations with an improved set of
  approximate eigenvectors", as in ARPACK / Krylov-Schur): when the basis holds `restart`
  blocks' worth of columns and the pairs have not converged, the basis becomes [Y, V_new] with Y = V U_p the
  lowest p = `keep` Ritz vectors (H Y = (H V) U_p by linearity, no product) and V_new the
  orthonormalised residual block the next iteration would have appended.  T = V^T H V is
  formed literally as before, so its Y rows hold the kept Ritz values and their couplings to
  V_new (the Krylov-Schur arrowhead); the residual estimate keeps its form.
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
    return theta, Uq[:, :nev], W, est, est_paper, Vb, HVb, th, Uq


def thick_restart(Vb, HVb, Uq, p, W):
    """The restarted basis blocks: ([Y, V_new], [H Y, None]) with Y = V U(:, 1:p), H Y = (H V) U(:, 1:p)
    and V R = W (CholQR2) the residual block; H V_new is left to the caller's next product."""
    Y = Vb @ Uq[:, :p]
    HY = HVb @ Uq[:, :p]
    Vn, _ = cholqr2(W)
    return [Y, Vn], [HY, None]


def block_lanczos(H, X0, nev, tol=1e-6, maxiter=200, U=None, stop=None, restart=None, keep=None):
    """stop(it, theta, relres) -> True ends the iteration early (used by the hybrid).
    restart: basis size, in blocks of nb columns, at which to restart (None: the basis grows
    without bound);
    keep: Ritz vectors kept at a restart (default: half the basis, at least nev)."""
    U = to_scipy_upper(H) if U is None else U
    V1, _ = cholqr2(np.asarray(X0, dtype=np.float64))
    Vs, HVs = [V1], [sym_upper_matmul(H, V1, U)]
    nb = V1.shape[1]
    hist = []
    theta, Uq, W, est, estp, Vb, HVb, th_all, Uq_all = _ritz(Vs, HVs, nev)
    hist.append(dict(it=0, theta=theta.copy(), relres=est.copy(), relres_paper=estp.copy(), basis=Vb.shape[1]))
    conv = bool(np.all(est < tol))
    it = 0
    spmm = 1
    restarts = 0
    while not conv and it < maxiter:
        if stop is not None and stop(it, theta, est):
            break
        it += 1
        try:
            if restart is not None and Vb.shape[1] >= restart * nb:
                p = keep if keep is not None else max(nev, (Vb.shape[1] // 2 // nb) * nb)
                Vs, HVs = thick_restart(Vb, HVb, Uq_all, p, W)
                Vn = Vs[-1]
                restarts += 1
            else:
                Vn, _ = cholqr2(W)
                Vs.append(Vn)
                HVs.append(None)
        except np.linalg.LinAlgError:
            break                                   # W rank deficient: basis exhausted
        HVs[-1] = sym_upper_matmul(H, Vn, U)
        spmm += 1
        theta, Uq, W, est, estp, Vb, HVb, th_all, Uq_all = _ritz(Vs, HVs, nev)
        hist.append(dict(it=it, theta=theta.copy(), relres=est.copy(), relres_paper=estp.copy(),
                         basis=Vb.shape[1]))
        conv = bool(np.all(est < tol))
    X = Vb @ Uq
    HX = HVb @ Uq
    return EigResult(theta=theta, X=X, relres=est, converged=conv, iterations=it, spmm=spmm,
                     spmv=spmm * nb, HX=HX, history=hist, extra=dict(restarts=restarts))
