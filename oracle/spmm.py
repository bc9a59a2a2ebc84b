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


class ParallelUpper:
    """U for sym_upper_matmul on several host threads: U and U^T (as CSR) cut in row ranges,
    each range's products in its own thread.  Every output row is the same sum, in the same
    order, as the single-threaded products (row i of U X over row i's entries; row j of U^T X
    over i ascending), so results are bitwise identical; only the wall time changes."""

    def __init__(self, U, threads):
        self.U = U
        self.threads = max(1, int(threads))
        Ut = U.T.tocsr()
        cuts = np.linspace(0, U.shape[0], self.threads + 1).astype(np.int64)
        self.parts = [(int(a), int(b), U[a:b], Ut[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
        self._d = U.diagonal()
        from concurrent.futures import ThreadPoolExecutor
        self.pool = ThreadPoolExecutor(self.threads)

    @property
    def shape(self):
        return self.U.shape

    def diagonal(self):
        return self._d

    def matmul(self, X):
        Y = np.empty((self.U.shape[0],) + X.shape[1:], dtype=np.float64)

        def run(part):
            a, b, Ua, Uta = part
            Y[a:b] = Ua @ X + Uta @ X

        list(self.pool.map(run, self.parts))
        return Y


def parallel_upper(H, threads):
    return ParallelUpper(to_scipy_upper(H), threads)


def sym_upper_matmul(H, X, U=None):
    """Y = (U + U^T - D) X in float64.  X: (n,) or (n, k).  U: scipy CSR of the upper triangle
    (built from H when None) or a ParallelUpper."""
    if U is None:
        U = to_scipy_upper(H)
    X = np.asarray(X, dtype=np.float64)
    d = U.diagonal()
    if isinstance(U, ParallelUpper):
        return U.matmul(X) - (d * X if X.ndim == 1 else d[:, None] * X)
    if X.ndim == 1:
        return U @ X + U.T @ X - d * X
    return U @ X + U.T @ X - d[:, None] * X


def spmv_count_per_spmm(k):
    """Sec. 2.6: an SpMM on k vectors counts as k SpMVs."""
    return int(k)
