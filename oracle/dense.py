"""Exact definition of the wanted result (oracle; test infrastructure only).

Sec. 2 (first paragraph): the n_ev algebraically smallest eigenvalues
lambda_1 <= ... <= lambda_nev of the symmetric H and their eigenvectors, H X = X Lambda
(Eq. eigen).  For n up to a few thousand this is a dense symmetric eigensolve.
"""
import numpy as np


def eigh_sorted(A):
    """All eigenpairs of a symmetric matrix, ascending (LAPACK syevd via numpy)."""
    A = np.asarray(A, dtype=np.float64)
    w, V = np.linalg.eigh(0.5 * (A + A.T))
    return w, V


def lowest_eigpairs(A, k):
    """The k algebraically smallest eigenpairs of dense symmetric A."""
    w, V = eigh_sorted(A)
    return w[:k].copy(), V[:, :k].copy()
