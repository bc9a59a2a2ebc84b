"""Hybrid block Lanczos / LOBPCG followed by batched RMM-DIIS (Sec. 2.8, Sec. 4) --
oracle, test infrastructure only.

The front method runs until the switching rule fires, then the n_ev lowest Ritz
vectors seed RMM-DIIS.  Switching rule: the average relative eigenvalue change
tau of Eq. (switchtau) falls to switch_tau (Sec. 4.1: 1e-7 for LOBPCG, 1e-4 for
block Lanczos with n_ev = 5), or -- the residual form used for the 2M-row
workload -- the largest relative residual of the wanted pairs falls to switch_res,
or a fixed number of front iterations has run (the sweeps of Tables 6-9).

Reading: when theta_j^(k) is below 1e-12 in magnitude its term in tau uses the
absolute change.

Option not in the paper (switch_gap): the switch also waits until every wanted Ritz pair has
||r_j|| <= switch_gap * gap_j, gap_j the distance to the block's nearest other Ritz value.  By
the Davis-Kahan bound each Ritz vector is then within that angle of its eigenvector; RMM-DIIS,
which has no orthogonalisation and converges to the eigenvector nearest its start (Sec. 3.3),
then starts inside the right eigenvector's basin rather than between near-degenerate ones.
"""
import numpy as np

from .block_lanczos import block_lanczos
from .lobpcg import lobpcg
from .result import EigResult
from .rmmdiis import rmmdiis
from .spmm import to_scipy_upper


def switch_tau(theta_k, theta_km1):
    """Eq. (switchtau): (1/n_ev) sqrt(sum_j ((theta_j^k - theta_j^{k-1}) / theta_j^k)^2)."""
    tk = np.asarray(theta_k, dtype=np.float64)
    tp = np.asarray(theta_km1, dtype=np.float64)
    den = np.where(np.abs(tk) < 1e-12, 1.0, tk)
    return float(np.sqrt(np.sum(((tk - tp) / den) ** 2)) / tk.size)


def gap_condition(theta, relres, nev, xi):
    """True when ||r_j|| <= xi * gap_j for every wanted pair j < nev, gap_j the distance from
    theta_j to the nearest other Ritz value of the block (Davis-Kahan: sin angle(z_j, v_j) <=
    ||r_j|| / gap_j).  theta ascending, relres = ||r_j|| / |theta_j|."""
    th = np.asarray(theta, dtype=np.float64)
    rn = np.asarray(relres, dtype=np.float64) * np.abs(th)
    for j in range(nev):
        gap = np.inf
        if j > 0:
            gap = min(gap, th[j] - th[j - 1])
        if j + 1 < th.size:
            gap = min(gap, th[j + 1] - th[j])
        if rn[j] > xi * gap:
            return False
    return True


def hybrid(H, X0, nev, tol=1e-6, front="lobpcg", switch_res=None, switch_tau_tol=1e-7,
           switch_after=None, front_maxiter=200, rmm_maxiter=200, s_max=10, precond="jacobi", U=None,
           rmm_precond="none", switch_gap=None):
    U = to_scipy_upper(H) if U is None else U
    state = dict(prev=None, taus=[], why=None)

    def stop(it, theta, relres):
        th = np.asarray(theta)[:nev]
        tau = switch_tau(th, state["prev"]) if state["prev"] is not None else np.inf
        state["prev"] = th.copy()
        state["taus"].append(tau)
        if switch_after is not None:
            if it >= switch_after:
                state["why"] = "after"
                return True
            return False
        if switch_gap is not None and not gap_condition(theta, relres, nev, switch_gap):
            return False
        if switch_res is not None and np.max(np.asarray(relres)[:nev]) <= switch_res:
            state["why"] = "res"
            return True
        if switch_tau_tol is not None and tau <= switch_tau_tol:
            state["why"] = "tau"
            return True
        return False

    if front == "lobpcg":
        fr = lobpcg(H, X0, nev, tol=tol, maxiter=front_maxiter, precond=precond, U=U, stop=stop)
    elif front == "block_lanczos":
        fr = block_lanczos(H, X0, nev, tol=tol, maxiter=front_maxiter, U=U, stop=stop)
    else:
        raise ValueError(front)
    if fr.converged:
        return EigResult(theta=fr.theta[:nev], X=fr.X[:, :nev], relres=fr.relres[:nev], converged=True,
                         iterations=fr.iterations, spmm=fr.spmm, spmv=fr.spmv, history=fr.history,
                         extra=dict(front=fr, rmm=None, switch=None, taus=state["taus"]))
    rm = rmmdiis(H, fr.X[:, :nev], tol=tol, maxiter=rmm_maxiter, s_max=s_max, HX0=fr.HX[:, :nev], U=U,
                 precond=rmm_precond)
    return EigResult(theta=rm.theta, X=rm.X, relres=rm.relres, converged=rm.converged,
                     iterations=fr.iterations + rm.iterations, spmm=fr.spmm + rm.spmm, spmv=fr.spmv + rm.spmv,
                     HX=rm.HX, history=fr.history + rm.history,
                     extra=dict(front=fr, rmm=rm, switch=state["why"], taus=state["taus"],
                                front_iterations=fr.iterations))
