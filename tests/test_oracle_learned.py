"""Pins of the learned-preconditioner oracle (oracle/learned.py) against closed forms, a
hand-worked example, central finite differences, brute force and the Jacobi-Davidson
correction equation solved densely."""
import numpy as np
import pytest

import oracle as O
from oracle import learned as L
from gen import CSRUpper, ci_matrix


def _tiny_H():
    """H = [[2, 1, 0], [1, -3, 0.5], [0, 0.5, 4]] as its upper triangle."""
    return CSRUpper(n=3, rowptr=np.array([0, 2, 4, 5], np.int64), col=np.array([0, 1, 1, 2, 2], np.int32),
                    val=np.array([2.0, 1.0, -3.0, 0.5, 4.0]), storage="f64")


def test_features_hand_worked():
    H = _tiny_H()
    R = np.array([[1.0], [2.0], [-2.0]])   # ||r|| = 3, sqrt(n) / ||r|| = sqrt(3) / 3
    F = L.features(H, [1.0], R)
    s = np.sqrt(3.0) / 3.0
    # (H - D) r = [1*2, 1*1 + 0.5*(-2), 0.5*2] = [2, 0, 1]
    want = np.array([[2.0, 1.0, 1.0, 3.0, 1.0 * s, 2.0 * s],
                     [-3.0, 1.0, -4.0, 4.5, 2.0 * s, 0.0],
                     [4.0, 1.0, 3.0, 4.5, -2.0 * s, 1.0 * s]])
    np.testing.assert_allclose(F[:, 0, :], want, rtol=0, atol=1e-15)
    # a zero residual column has zero residual features
    F0 = L.features(H, [1.0, 2.0], np.c_[R, np.zeros(3)])
    assert np.all(F0[:, 1, 4:] == 0) and np.all(F0[:, 1, 2] == np.array([0.0, -5.0, 2.0]))


def test_row_abs_sum_brute_force():
    H = ci_matrix(400, 40, 64, seed=3, storage="f64")
    D = O.to_dense(H)
    np.testing.assert_allclose(L.row_abs_sum(H), np.abs(D).sum(axis=1), rtol=1e-14, atol=1e-14)


def test_jacobi_scale():
    np.testing.assert_array_equal(L.jacobi_scale([0.0, 1.0, -1.5, 4.0, -8.0]), [0.5, 0.5, -0.5, 0.25, -0.125])


def test_forward_closed_form_linear_network():
    """Hidden units relu(u_k), relu(-u_k) recombined with +-c_k give o = c . u + b3 exactly, and
    m = J(f2) (1 + o)."""
    rng = np.random.default_rng(0)
    mu, sg = rng.standard_normal(6), 0.5 + rng.random(6)
    c = rng.standard_normal(6)
    W1 = np.zeros((32, 6)); W2 = np.zeros((32, 32)); w3 = np.zeros(32)
    for k in range(6):
        W1[k, k], W1[6 + k, k] = 1.0, -1.0
        w3[k], w3[6 + k] = c[k], -c[k]
    W2[:12, :12] = np.eye(12)
    p = L.pack(dict(mu=mu, sigma=sg, W1=W1, b1=np.zeros(32), W2=W2, b2=np.zeros(32), w3=w3, b3=0.25))
    F = rng.standard_normal((7, 3, 6)) * 3
    m, _ = L.forward(p, F)
    J = 1.0 / np.where(F[..., 2] < 0, -1, 1) / np.maximum(np.abs(F[..., 2]), 2.0)
    np.testing.assert_allclose(m, J * (1.0 + ((F - mu) / sg) @ c + 0.25), rtol=1e-13, atol=1e-13)
    # zero output layer: exactly the Jacobi scale
    p[L.OFF_W3:L.OFF_B3 + 1] = 0.0
    np.testing.assert_array_equal(L.forward(p, F)[0], J)


def _random_problem(seed=1, n=12, m=3):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(L.N_PARAMS) * 0.4
    p[L.OFF_MU:L.OFF_MU + 6] = rng.standard_normal(6) * 0.1
    p[L.OFF_SIGMA:L.OFF_SIGMA + 6] = 0.5 + rng.random(6)
    F = rng.standard_normal((n, m, 6))
    R = rng.standard_normal((n, m))
    Z = rng.standard_normal((n, m))
    c = np.array([0.7, 0.0, 1.3])[:m]
    return p, F, R, Z, c


def test_backward_central_differences():
    p, F, R, Z, c = _random_problem()
    _, g = L.loss_grad(p, F, R, Z, c)
    assert np.all(g[:L.N_FIXED] == 0)
    h = 1e-6
    fd = np.zeros(L.N_PARAMS)
    for q in range(L.N_FIXED, L.N_PARAMS):
        pp, pm = p.copy(), p.copy()
        pp[q] += h
        pm[q] -= h
        fd[q] = (L.loss(pp, F, R, Z, c)[0] - L.loss(pm, F, R, Z, c)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=0, atol=2e-7 * max(1.0, np.abs(g).max()))
    # every parameter block receives gradient
    for a, b in [(L.OFF_W1, L.OFF_B1), (L.OFF_B1, L.OFF_W2), (L.OFF_W2, L.OFF_B2), (L.OFF_B2, L.OFF_W3),
                 (L.OFF_W3, L.OFF_B3), (L.OFF_B3, L.N_PARAMS)]:
        assert np.abs(g[a:b]).max() > 0


def test_loss_zero_at_its_minimum():
    p, F, R, _, c = _random_problem(seed=2)
    m, _ = L.forward(p, F)
    val, g = L.loss_grad(p, F, R, m * R, c)
    assert val == 0.0 and np.all(g == 0)


def test_loss_column_weighting():
    """One column, f2 = 0 (J = 1/2) and b3 = 1, so m = 1: L = sum((r - z)^2) / ||z||^2."""
    p = np.zeros(L.N_PARAMS)
    p[L.OFF_SIGMA:L.OFF_SIGMA + 6] = 1.0
    p[L.OFF_B3] = 1.0
    F = np.zeros((3, 1, 6))
    R = np.array([[2.0], [0.0], [-4.0]])
    Z = np.array([[1.0], [1.0], [1.0]])
    c = np.array([1.0 / (Z[:, 0] @ Z[:, 0])])
    val = L.loss(p, F, R, Z, c)[0]
    assert val == pytest.approx(((2 - 1) ** 2 + (0 - 1) ** 2 + (-4 - 1) ** 2) / 3.0, rel=1e-15)


def test_correction_target_diagonal_closed_form():
    n = 6
    Xs = np.eye(n)[:, :2]
    x = np.zeros(n); x[0], x[3] = 1.0, 0.1
    x /= np.linalg.norm(x)
    Z, c = L.correction_target(x[:, None], Xs)
    want = x.copy(); want[0] = x[0] - 1.0 / x[0]
    np.testing.assert_allclose(Z[:, 0], want, rtol=0, atol=1e-15)
    assert c[0] == pytest.approx(1.0 / (want @ want), rel=1e-14)
    # x orthogonal to X*: no target (weight 0)
    Z2, c2 = L.correction_target(np.eye(n)[:, 4:5], Xs)
    assert c2[0] == 0 and np.all(Z2 == 0)


def test_correction_target_orthogonal_to_x():
    rng = np.random.default_rng(5)
    Xs = np.linalg.qr(rng.standard_normal((50, 4)))[0]
    X = Xs @ rng.standard_normal((4, 3)) + 0.05 * rng.standard_normal((50, 3))
    X /= np.linalg.norm(X, axis=0)
    Z, c = L.correction_target(X, Xs)
    np.testing.assert_allclose((Z * X).sum(axis=0), 0, atol=1e-14)
    assert np.all(c > 0)


def _jd_correction(Hd, x):
    """Exact solution t of (I - xx^T)(H - theta I)(I - xx^T) t = -r, t orthogonal to x (dense)."""
    n = x.size
    th = x @ Hd @ x
    r = Hd @ x - th * x
    Q = np.linalg.qr(np.c_[x, np.eye(n)[:, : n - 1]])[0][:, 1:]   # orthonormal basis of x-perp
    y = np.linalg.solve(Q.T @ (Hd - th * np.eye(n)) @ Q, -(Q.T @ r))
    return Q @ y


def test_correction_target_is_the_jacobi_davidson_correction_to_second_order():
    """z = -t + O(eps^2) relative, t the exact projected correction of Jacobi-Davidson."""
    rng = np.random.default_rng(7)
    n = 30
    A = rng.standard_normal((n, n)) * 0.1
    Hd = (A + A.T) / 2 + np.diag(np.arange(n, dtype=float))
    w, V = np.linalg.eigh(Hd)
    xs = V[:, 0]
    e = rng.standard_normal(n); e -= (e @ xs) * xs; e /= np.linalg.norm(e)
    errs = []
    for eps in (1e-2, 1e-3):
        x = xs + eps * e
        x /= np.linalg.norm(x)
        Z, _ = L.correction_target(x[:, None], xs[:, None])
        t = _jd_correction(Hd, x)
        errs.append(np.linalg.norm(Z[:, 0] + t) / np.linalg.norm(Z[:, 0]))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 30, errs


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(L.N_PARAMS)
    g = rng.standard_normal(L.N_PARAMS)
    lr, eps = 1e-3, 1e-8
    p1, m1, m2 = L.adam_step(p, g, np.zeros(L.N_PARAMS), np.zeros(L.N_PARAMS), 1, lr, eps=eps)
    want = p - lr * g / (np.abs(g) + eps)
    want[:L.N_FIXED] = p[:L.N_FIXED]
    np.testing.assert_allclose(p1, want, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1[L.N_FIXED:], 0.1 * g[L.N_FIXED:], rtol=1e-14)
    np.testing.assert_allclose(m2[L.N_FIXED:], 0.001 * g[L.N_FIXED:] ** 2, rtol=1e-12)


def test_apply_falls_back_to_jacobi_on_non_finite():
    H = _tiny_H()
    R = np.array([[1.0, 0.5], [2.0, -1.0], [-2.0, 3.0]])
    th = [1.0, -2.9]
    F = L.features(H, th, R)
    p = np.zeros(L.N_PARAMS)
    p[L.OFF_SIGMA:L.OFF_SIGMA + 6] = 1.0
    p[L.OFF_B3] = np.nan
    np.testing.assert_array_equal(L.apply(p, F, R, H.diagonal_f64(), th), O.jacobi_apply(H.diagonal_f64(), th, R))
    p[L.OFF_B3] = 0.5
    np.testing.assert_allclose(L.apply(p, F, R, H.diagonal_f64(), th),
                               1.5 * O.jacobi_apply(H.diagonal_f64(), th, R, 2.0), rtol=1e-15)


def test_oracle_training_improves_on_jacobi():
    """The whole recipe in FP64 on a small family: samples from perturbed eigenvectors, the
    network started as the Jacobi K (zero output layer), Adam on the loss gradient; the training
    loss falls below the Jacobi K's."""
    from gen import family_perturbation, family_member
    H0 = ci_matrix(600, 60, 64, seed=11, storage="f64")
    V = family_perturbation(H0, seed=12)
    rng = np.random.default_rng(13)
    samples = []
    for g in (0.6, 0.9, 1.2):
        H = family_member(H0, V, g)
        D = O.to_dense(H)
        w, Z = np.linalg.eigh(D)
        Xs = Z[:, :6]
        X = np.linalg.qr(Xs + 0.05 * rng.standard_normal(Xs.shape))[0]
        th = np.einsum("ij,ij->j", X, D @ X)
        R = L.residual(H, X, th)
        F = L.features(H, th, R)
        Zt, c = L.correction_target(X, Xs)
        samples.append((F, R, Zt, c))
    Fall = np.concatenate([s[0].reshape(-1, 6) for s in samples])
    p = np.zeros(L.N_PARAMS)
    p[0:6], p[6:12] = Fall.mean(axis=0), np.maximum(Fall.std(axis=0), 1e-6)
    p[L.OFF_W1:L.OFF_B1] = rng.standard_normal(192) * np.sqrt(2 / 6)
    p[L.OFF_W2:L.OFF_B2] = rng.standard_normal(1024) * np.sqrt(2 / 32)
    jac = np.mean([L.loss(p, *s)[0] for s in samples])          # zero output layer: the Jacobi K
    jac_direct = np.mean([((R * L.jacobi_scale(F[..., 2]) - Zt) ** 2 * c).sum() / (c > 0).sum()
                          for F, R, Zt, c in samples])
    assert jac == pytest.approx(jac_direct, rel=1e-12)
    m1, m2 = np.zeros(L.N_PARAMS), np.zeros(L.N_PARAMS)
    t = 0
    for ep in range(60):
        for s in samples:
            t += 1
            _, g = L.loss_grad(p, *s)
            p, m1, m2 = L.adam_step(p, g, m1, m2, t, 3e-3)
    trained = np.mean([L.loss(p, *s)[0] for s in samples])
    assert trained < 0.9 * jac, (trained, jac)
