"""Pins for ChebFSI (Alg. 3), RMM-DIIS (Alg. 4) and the hybrid switch (Eq. switchtau)."""
import os

import numpy as np
import pytest

import oracle as O
from gen import (laplacian_kron, laplacian_kron_eigs, diagonal_matrix, ci_matrix, random_block,
                 principal_submatrix, pad_rows)


def cheb_scalar(m, t):
    """T_m(t) = cos(m arccos t) on [-1, 1] and cosh(m arccosh |t|) (with sign (-1)^m for t < -1)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1
    out[inside] = np.cos(m * np.arccos(t[inside]))
    o = ~inside
    out[o] = np.cosh(m * np.arccosh(np.abs(t[o]))) * np.where(t[o] < 0, (-1.0) ** m, 1.0)
    return out


@pytest.mark.parametrize("deg", [1, 2, 5, 10, 24])
def test_cheb_filter_diagonal_matches_scalar(deg):
    d = np.linspace(-1.5, 9.0, 40)
    H = diagonal_matrix(d)
    c, e = 4.0, 3.0
    Q = np.eye(40)[:, :40]
    Y, prods = O.cheb_filter(H, Q, O.sym_upper_matmul(H, Q), deg, c, e)
    assert prods == deg - 1
    np.testing.assert_allclose(np.diag(Y), cheb_scalar(deg, (d - c) / e), rtol=1e-12, atol=1e-12)


def test_cheb_filter_locked_columns_untouched():
    d = np.linspace(0, 5, 10)
    H = diagonal_matrix(d)
    Q = np.eye(10)
    act = np.array([True] * 5 + [False] * 5)
    Y, _ = O.cheb_filter(H, Q, O.sym_upper_matmul(H, Q), 6, 3.0, 2.0, act)
    np.testing.assert_array_equal(Y[:, 5:], Q[:, 5:])


def test_lambda_ub_and_chebfsi_laplacian():
    dims = [9, 11, 13]
    H = laplacian_kron(dims)
    exact = laplacian_kron_eigs(dims)
    lub, k = O.lambda_ub_estimate(H, random_block(H.n, 1, 3)[:, 0])
    assert k == 10
    assert exact[-1] <= lub <= exact[-1] * 1.2
    r = O.chebfsi(H, random_block(H.n, 8, 5), 5, deg=10, tol=1e-8, v_ub=random_block(H.n, 1, 3)[:, 0])
    assert r.converged
    np.testing.assert_allclose(r.theta, exact[:5], rtol=1e-10)


def test_rr2_closed_form():
    rng = np.random.default_rng(0)
    A0 = rng.standard_normal((30, 30)); A0 = A0 + A0.T
    x, r = rng.standard_normal(30), rng.standard_normal(30)
    Hx, Hr = A0 @ x, A0 @ r
    th, g = O.rr2(x, r, Hx, Hr)
    a11, a12, a22 = x @ Hx, x @ Hr, r @ Hr
    b11, b12, b22 = x @ x, x @ r, r @ r
    qa = b11 * b22 - b12 ** 2
    qb = -(a11 * b22 + a22 * b11 - 2 * a12 * b12)
    qc = a11 * a22 - a12 ** 2
    root = (-qb - np.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
    assert abs(th - root) < 1e-10 * abs(root)
    w = g[0] * x + g[1] * r
    assert abs(w @ w - 1) < 1e-12
    assert g[0] <= 0


def test_diis_two_vector_closed_form():
    rng = np.random.default_rng(1)
    r1, r2 = rng.standard_normal(50), rng.standard_normal(50)
    a = O.diis_coefficients([r1, r2])
    a_old = (r2 @ (r2 - r1)) / ((r2 - r1) @ (r2 - r1))
    np.testing.assert_allclose(a, [a_old, 1 - a_old], rtol=1e-12)
    assert O.diis_coefficients([r1]).tolist() == [1.0]


def test_rmmdiis_fixed_point_and_convergence():
    dims = [9, 10, 11]
    H = laplacian_kron(dims)
    lam, V = O.lowest_eigpairs(O.to_dense(H), 3)
    r = O.rmmdiis(H, V, tol=1e-10)
    assert r.converged and r.iterations == 0
    X0 = V + 1e-3 * random_block(H.n, 3, 7)
    r = O.rmmdiis(H, X0, tol=1e-9, maxiter=400, s_max=20)
    assert r.converged
    np.testing.assert_allclose(r.theta, lam, rtol=1e-10)
    assert np.all(O.true_relres(H, r.theta, r.X) < 1e-8)


def test_switch_tau_hand_value():
    # changes: (1.0-1.1)/1.0 = -0.1, (2.0-2.2)/2.0 = -0.1 -> sqrt(0.02)/2 = 0.0707106781...
    assert abs(O.switch_tau([1.0, 2.0], [1.1, 2.2]) - 0.07071067811865475) < 1e-15
    assert O.switch_tau([3.0, 4.0], [3.0, 4.0]) == 0.0


def test_gap_condition_hand_values():
    """||r_j|| <= xi * gap_j by hand: theta = (1.0, 1.1, 2.0), relres = (1e-3, 1e-2, 1e-3):
    ||r|| = (1e-3, 1.1e-2, 2e-3), gaps (0.1, 0.1, 0.9).  With xi = 0.2 pair 1 needs 1.1e-2 <= 0.02:
    true; with xi = 0.1, 1.1e-2 <= 0.01 fails.  Only the wanted pairs count (nev = 1 passes at
    xi = 0.02: 1e-3 <= 0.002)."""
    th, rel = [1.0, 1.1, 2.0], [1e-3, 1e-2, 1e-3]
    assert O.gap_condition(th, rel, 3, 0.2)
    assert not O.gap_condition(th, rel, 3, 0.1)
    assert O.gap_condition(th, rel, 1, 0.02)
    assert not O.gap_condition(th, rel, 1, 0.009)


def test_hybrid_gap_switch_converges_on_the_cut_shell():
    """With the gap condition (not in the paper) the oracle's hybrid switches once the wanted
    Ritz vectors are separated from their neighbours and its RMM-DIIS converges to the dense
    spectrum's lowest pairs."""
    H = ci_matrix(3000, 100, 64, seed=1, storage="f64")
    lam, _ = O.lowest_eigpairs(O.to_dense(H), 8)
    X0 = pad_rows(O.lowest_eigpairs(O.to_dense(principal_submatrix(H, 300)), 16)[1], H.n)
    r = O.hybrid(H, X0, 8, tol=1e-6, switch_res=1e-2, switch_tau_tol=None, switch_gap=0.03, rmm_maxiter=200,
                 rmm_precond="jacobi")
    assert r.converged
    np.testing.assert_allclose(np.sort(r.theta), lam, rtol=1e-9)
    fr = r.extra["front"]
    last = fr.history[-1]
    assert O.gap_condition(last["theta"], last["relres"], 8, 0.03) or r.extra["rmm"] is None


def test_hybrid_ci_vs_dense():
    H = ci_matrix(3000, 100, 64, seed=1, storage="f64")
    lam, _ = O.lowest_eigpairs(O.to_dense(H), 5)
    Z0 = O.lowest_eigpairs(O.to_dense(principal_submatrix(H, 300)), 8)[1]
    X0 = pad_rows(Z0, H.n)
    for front, tau in [("lobpcg", 1e-7), ("block_lanczos", 1e-7)]:
        r = O.hybrid(H, X0, 5, tol=1e-6, front=front, switch_tau_tol=tau, rmm_maxiter=400)
        assert r.converged, front
        np.testing.assert_allclose(r.theta, lam, rtol=1e-9)
        assert np.all(O.true_relres(H, r.theta, r.X) < 1e-6)
    r = O.hybrid(H, X0, 5, tol=1e-6, switch_after=3, switch_tau_tol=None, rmm_maxiter=400)
    assert r.extra["front_iterations"] == 3 and r.extra["switch"] == "after"


def _window_fixture():
    path = os.path.join(os.path.dirname(__file__), "golden", "rmmdiis_window.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    xs = [np.array([1.0, 0.0]), np.array([0.0, 1.0]), np.array([1.0, 1.0])]
    rs = [np.array([1.0, 1.0]), np.array([1.0, 0.0]), np.array([0.0, 2.0])]
    return xs, rs, [(int(r[0]), np.array([float(r[1]), float(r[2])])) for r in rows]


def check_diis_window():
    """tests/golden/rmmdiis_window.txt: x~ of Eq. (xsum) over the newest s iterates, worked by
    hand for s_max = 1, 2, 3 on three two-dimensional histories."""
    xs, rs, want = _window_fixture()
    for s_max, xt in want:
        np.testing.assert_allclose(O.diis_extrapolate(xs, rs, s_max), xt, rtol=0, atol=1e-14)


def test_diis_window_hand_worked():
    check_diis_window()


def check_cheb_filter_diagonal(deg=5):
    d = np.linspace(-1.5, 9.0, 40)
    H = diagonal_matrix(d)
    c, e = 4.0, 3.0
    Q = np.eye(40)
    Y, _ = O.cheb_filter(H, Q, O.sym_upper_matmul(H, Q), deg, c, e)
    np.testing.assert_allclose(np.diag(Y), cheb_scalar(deg, (d - c) / e), rtol=1e-12, atol=1e-12)


def check_diis_two_vector():
    rng = np.random.default_rng(1)
    r1, r2 = rng.standard_normal(50), rng.standard_normal(50)
    a_old = (r2 @ (r2 - r1)) / ((r2 - r1) @ (r2 - r1))
    np.testing.assert_allclose(O.diis_coefficients([r1, r2]), [a_old, 1 - a_old], rtol=1e-12)


def check_rmmdiis_converges_to_lowest():
    H = laplacian_kron([9, 10, 11])
    lam, V = O.lowest_eigpairs(O.to_dense(H), 3)
    r = O.rmmdiis(H, V + 1e-3 * random_block(H.n, 3, 7), tol=1e-9, maxiter=400, s_max=20)
    assert r.converged
    np.testing.assert_allclose(r.theta, lam, rtol=1e-10)


def test_planted_mistakes_are_caught(monkeypatch):
    """Mistakes planted in the oracle itself (its module functions replaced by wrong variants)
    fail the pins above: a recurrence with + Q_prev (Eq. chebypoly), a DIIS window over the
    oldest instead of the newest iterates, DIIS coefficients without the affine constraint of
    Eq. (alphasum), and the larger root of the 2x2 pencil (Eq. rr)."""
    import importlib
    C = importlib.import_module("oracle.chebfsi")   # the modules (the package re-exports functions
    R = importlib.import_module("oracle.rmmdiis")   # of the same names)
    check_cheb_filter_diagonal()
    check_diis_window()
    check_diis_two_vector()
    check_rmmdiis_converges_to_lowest()

    with monkeypatch.context() as m:
        m.setattr(C, "cheb_step", lambda HW, W, Qp, c, e: 2.0 * (HW - c * W) / e + Qp)
        with pytest.raises(AssertionError):
            check_cheb_filter_diagonal()

    def oldest_window(xs, rs, s_max):
        s = min(len(xs), s_max)
        alpha = R.diis_coefficients(rs[:s])
        xt = sum(al * xv for al, xv in zip(alpha, xs[:s]))
        return xt / np.linalg.norm(xt)
    with monkeypatch.context() as m:
        m.setattr(R, "diis_extrapolate", oldest_window)
        m.setattr(O, "diis_extrapolate", oldest_window)
        with pytest.raises(AssertionError):
            check_diis_window()

    def unconstrained(rs):
        A = np.stack([np.asarray(r, dtype=np.float64) for r in rs], axis=1)
        a, *_ = np.linalg.lstsq(A, A[:, -1], rcond=None)   # fits the newest residual instead
        return a
    with monkeypatch.context() as m:
        m.setattr(R, "diis_coefficients", unconstrained)
        m.setattr(O, "diis_coefficients", unconstrained)
        with pytest.raises(AssertionError):
            check_diis_two_vector()
        with pytest.raises(AssertionError):
            check_diis_window()

    real_rr2 = R.rr2

    def larger_root(x, r, Hx, Hr):
        A = np.array([[x @ Hx, x @ Hr], [r @ Hx, r @ Hr]])
        B = np.array([[x @ x, x @ r], [r @ x, r @ r]])
        import scipy.linalg as sla
        w, G = sla.eigh(0.5 * (A + A.T), 0.5 * (B + B.T))
        return float(w[1]), G[:, 1]
    with monkeypatch.context() as m:
        m.setattr(R, "rr2", larger_root)
        with pytest.raises(AssertionError):
            check_rmmdiis_converges_to_lowest()
    assert R.rr2 is real_rr2


def test_certification_bounds_contain_the_exact_eigenvalue():
    """Residual bound |lambda - theta| <= ||r|| and Kato-Temple |lambda - theta| <= ||r||^2 / gap
    (gap to the rest of the spectrum) for Rayleigh quotients of perturbed eigenvectors, against the
    dense spectrum."""
    H = ci_matrix(400, 40, 64, seed=8, storage="f64")
    D = O.to_dense(H)
    w, V = np.linalg.eigh(D)
    rng = np.random.default_rng(2)
    for j, eps in [(0, 1e-3), (3, 1e-2), (7, 1e-4)]:
        z = V[:, j] + eps * rng.standard_normal(H.n)
        z /= np.linalg.norm(z)
        th = z @ D @ z
        rn = O.residual_bound(H, np.array([th]), z[:, None])[0]
        assert rn == pytest.approx(np.linalg.norm(D @ z - th * z), rel=1e-10)
        k = np.argmin(np.abs(w - th))
        assert abs(w[k] - th) <= rn * (1 + 1e-12)
        gap = np.min(np.abs(np.delete(w, k) - th))
        assert abs(w[k] - th) <= O.kato_temple(rn, gap) * (1 + 1e-9)


def test_missed_eigenvalue_guard():
    """Lanczos from three random starts confirms a correct lowest-five result and finds the
    eigenvalue a planted mistake left out (a result holding lambda_1, lambda_3..lambda_6)."""
    H = ci_matrix(1500, 60, 64, seed=4, storage="f64")
    w = np.linalg.eigvalsh(O.to_dense(H))
    assert O.missed_eigenvalues(H, w[:5], 5).size == 0
    missed = O.missed_eigenvalues(H, np.r_[w[0], w[2:6]], 5)
    assert missed.size >= 1 and np.min(np.abs(missed - w[1])) < 1e-8 * np.abs(w[:6]).max()
