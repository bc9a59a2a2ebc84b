"""Preconditioner K^{-1} of Eq. (wblock) (oracle; test infrastructure only).

The paper only says K "approximates H in some way" (Sec. 2.3).  The reading used
throughout this project is the diagonal (Jacobi) preconditioner
    w_ij = r_ij / (H_ii - theta_j),
with the denominator's magnitude floored at `floor` (sign kept, zero -> +floor),
so that rows whose diagonal is close to the Ritz value are not amplified without
bound.  The floor is a documented constant (0.1 by default; the synthetic level
spacing is 1).
"""
import numpy as np


def jacobi_apply(diagH, theta, R, floor=0.1):
    diagH = np.asarray(diagH, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    den = diagH[:, None] - theta[None, :]
    mag = np.maximum(np.abs(den), floor)
    den = np.where(den < 0, -mag, mag)
    return np.asarray(R, dtype=np.float64) / den
