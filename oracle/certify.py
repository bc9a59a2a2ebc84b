"""Certification of approximate eigenpairs (oracle; test infrastructure only).

Relative residual norm of Sec. 3.2: ||H z - z theta|| / |theta|.  For symmetric H,
an eigenvalue lies within ||r|| of theta (residual bound), and within ||r||^2 / gap
when theta is separated by `gap` from the rest of the spectrum (Kato-Temple); both
are textbook bounds (Parlett, The Symmetric Eigenvalue Problem, Ch. 4 and 10).
"""
import numpy as np

from .spmm import sym_upper_matmul


def true_relres(H, theta, Z, U=None):
    """Per-column ||H z_j - theta_j z_j|| / |theta_j| with z_j normalised, float64."""
    Z = np.asarray(Z, dtype=np.float64)
    Z = Z / np.linalg.norm(Z, axis=0, keepdims=True)
    HZ = sym_upper_matmul(H, Z, U)
    theta = np.asarray(theta, dtype=np.float64)
    R = HZ - Z * theta[None, :]
    return np.linalg.norm(R, axis=0) / np.abs(theta)


def residual_bound(H, theta, Z, U=None):
    """||r_j|| with z_j normalised: some eigenvalue lies in [theta - ||r||, theta + ||r||]."""
    return true_relres(H, theta, Z, U) * np.abs(theta)


def kato_temple(rnorm, gap):
    """Kato-Temple eigenvalue error bound ||r||^2 / gap."""
    return np.asarray(rnorm) ** 2 / np.asarray(gap)


def missed_eigenvalues(H, theta, nev, starts=3, tol=1e-10, seed=0, U=None, rel_gap=1e-8):
    """Guard against a result that skipped a wanted eigenvalue (a method that converged to
    interior pairs): Lanczos with full reorthogonalisation (Sec. 2.1) from `starts` seeded random
    vectors, to relative residual `tol`; returns the eigenvalues it finds at or below
    max(theta) that match no entry of theta to rel_gap (relative to max |theta|).  An empty
    array means no wanted eigenvalue is missing, up to the multiplicity a single-vector Krylov
    space can see (a multiple eigenvalue shows up once per start)."""
    from .lanczos import lanczos
    theta = np.sort(np.asarray(theta, dtype=np.float64))
    top = theta.max()
    scale = max(np.abs(theta).max(), 1e-300)
    rng = np.random.default_rng(seed)
    missed = []
    for _ in range(starts):
        r = lanczos(H, rng.standard_normal(H.n), nev, tol=tol, U=U)
        for lam in np.sort(r.theta[:nev]):
            if lam <= top + rel_gap * scale and np.min(np.abs(theta - lam)) > rel_gap * scale:
                missed.append(lam)
    return np.unique(np.round(np.asarray(missed), 12))
