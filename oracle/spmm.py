"""Y = H X for symmetric H stored as its upper triangle (oracle; test infrastructure only).

Sec. 3.1 (Tables 2-3) counts nonzeros "in half the symmetric matrices": only the
upper triangle U (incl. diagonal D) is stored, and H = U + U^T - D.  The SpMM of
Sec. 1 / Eqs. (upd1)-(upd2) is therefore Y = U X + U^T X - D X, which is the
definition written out below with scipy's sparse products as the primitive.
"""
import numpy as np
import scipy.sparse as sp


def to_scipy_upper(H):
    """scipy CSR of the stored upper triangle U (float64 values)."""
    return sp.csr_matrix((H.values_f64(), H.col.astype(np.int64), H.rowptr), shape=(H.n, H.n))


def to_dense(H):
    """Dense symmetric H = U + U^T - D (small n only)."""
    U = to_scipy_upper(H).toarray()
    return U + U.T - np.diag(np.diag(U))


def sym_upper_matmul(H, X, U=None):
    """Y = (U + U^T - D) X in float64.  X: (n,) or (n, k)."""
    if U is None:
        U = to_scipy_upper(H)
    X = np.asarray(X, dtype=np.float64)
    d = U.diagonal()
    if X.ndim == 1:
        return U @ X + U.T @ X - d * X
    return U @ X + U.T @ X - d[:, None] * X


def spmv_count_per_spmm(k):
    """Sec. 2.6: an SpMM on k vectors counts as k SpMVs."""
    return int(k)
