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
