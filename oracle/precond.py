"""Preconditioner K^{-1} of Eq. (wblock) (oracle; test infrastructure only).

The paper only says K "approximates H in some way" (Sec. 2.3).  The reading used
throughout this project is the diagonal (Jacobi) preconditioner
    w_ij = r_ij / (H_ii - theta_j),
with the denominator's magnitude floored at `floor` (sign kept, zero -> +floor),
so that rows whose diagonal is close to the Ritz value are not amplified.  The
floor is a documented constant: 2.0 by default, i.e. two level spacings of the
CI-shaped spectrum (spacing 1), so that the rows of a wanted vector's near-degenerate
shell neighbours are not amplified over the rest while high-energy rows are still
damped by 1/(H_ii - theta).
"""
import numpy as np


def jacobi_apply(diagH, theta, R, floor=2.0):
    diagH = np.asarray(diagH, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    den = diagH[:, None] - theta[None, :]
    mag = np.maximum(np.abs(den), floor)
    den = np.where(den < 0, -mag, mag)
    return np.asarray(R, dtype=np.float64) / den
