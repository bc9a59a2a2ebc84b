"""Pins for the exact definition (Sec. 2: the n_ev smallest eigenpairs)."""
import numpy as np

import oracle as O
from gen import laplacian_kron, laplacian_kron_eigs, diagonal_matrix


def test_laplacian_closed_form_spectrum():
    dims = [5, 6, 7]
    H = laplacian_kron(dims)
    lam, V = O.lowest_eigpairs(O.to_dense(H), 12)
    np.testing.assert_allclose(lam, laplacian_kron_eigs(dims)[:12], rtol=0, atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(12), atol=1e-12)


def test_diagonal():
    d = np.array([3.0, -1.0, 2.0, 0.5])
    lam, V = O.lowest_eigpairs(O.to_dense(diagonal_matrix(d)), 2)
    np.testing.assert_array_equal(lam, [-1.0, 0.5])
    assert abs(abs(V[1, 0]) - 1) < 1e-15 and abs(abs(V[3, 1]) - 1) < 1e-15


def test_golden_tridiagonal():
    """tests/golden/tridiag4.txt: T_4 = tridiag(-1,2,-1) has eigenvalues 2 - 2cos(k pi / 5)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tridiag4.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    expect = np.array([float(r[0]) for r in rows])
    H = laplacian_kron([4])
    lam, _ = O.lowest_eigpairs(O.to_dense(H), 4)
    np.testing.assert_allclose(lam, expect, atol=1e-15)
