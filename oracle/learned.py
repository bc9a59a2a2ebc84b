"""Learned per-row preconditioner (oracle; TEST INFRASTRUCTURE ONLY).

The paper leaves K of Eq. (wblock) open: it only has to approximate H "in some way"
(Sec. 2.3), and Secs. 5-6 name better preconditioners as what would cut the iteration
counts further.  This module defines the learned replacement of the Jacobi K^{-1} that
the GPU path trains and applies, in plain float64 numpy, as the reference the CUDA
kernels are checked against.  Nothing here is tuned or blocked: each function is the
definition written out.

Preconditioned residual (one entry per row i and block column j)
    w_ij = m_ij * r_ij,        m_ij = MLP(standardise(f_ij)),
with six features of row i and column j
    f0 = H_ii                        f3 = (|H| 1)_i      (absolute row sum of the full H)
    f1 = theta_j                     f4 = sqrt(n) r_ij / ||r_j||
    f2 = H_ii - theta_j              f5 = sqrt(n) ((H - D) r_j)_i / ||r_j||
(f4 and f5 are zero for a zero column).  f5 is the one-hop aggregate of the residual:
the off-diagonal part of (H r_j)_i; the diagonal part is H_ii r_ij, already given by f0
and f4.  The two residual features are scaled to unit root-mean-square so that one
network serves every residual size from the start of a solve to convergence.

Network: 6 -> 32 -> 32 -> 1, ReLU after both hidden layers, linear output o; u = (f - mu) /
sigma with mu, sigma fixed (feature statistics of the training set).  The network learns a
correction of the Jacobi scale J = 1 / floor(f2) (magnitude floored at JACOBI_FLOOR = 2, sign
kept, zero -> +2, as oracle.precond):
    m = J (1 + o),
so that a zero output layer is exactly the Jacobi K.  A non-finite m r falls back to the
Jacobi value r / floor(H_ii - theta_j) with the solver's floor (oracle.precond).

Flat parameter vector (float32 on the GPU, the order the C ABI documents):
    mu[6] sigma[6] | W1[32][6] b1[32] W2[32][32] b2[32] w3[32] b3
The first 12 entries are fixed; the 1313 after them are trained.

Training target (reading of "(residual, (H - theta I)^{-1} r) pairs"): the Jacobi-Davidson
correction of x_j to first order.  With x = x* + e near an eigenvector x*,
r = (H - theta) e + O(|e|^2), so (H - theta)^{-1} r is the error e itself; measured
against the converged wanted subspace X* (orthonormal n x k) it is
    z_j = x_j - X* p / (p^T p),   p = X*^T x_j,
which is orthogonal to a unit x_j.  Loss of one sample (columns with a target)
    L = (1/|J|) sum_{j in J} sum_i (m_ij r_ij - z_ij)^2 / ||z_j||^2.
"""
import numpy as np
import scipy.sparse as sp

from .spmm import to_scipy_upper, sym_upper_matmul
from .precond import jacobi_apply

N_FEAT = 6
HIDDEN = 32
OFF_MU, OFF_SIGMA = 0, 6
OFF_W1 = 12
OFF_B1 = OFF_W1 + HIDDEN * N_FEAT
OFF_W2 = OFF_B1 + HIDDEN
OFF_B2 = OFF_W2 + HIDDEN * HIDDEN
OFF_W3 = OFF_B2 + HIDDEN
OFF_B3 = OFF_W3 + HIDDEN
N_PARAMS = OFF_B3 + 1          # 1325
N_FIXED = 12
JACOBI_FLOOR = 2.0


def jacobi_scale(f2):
    """J = 1 / floor(f2): |f2| floored at JACOBI_FLOOR, sign kept, zero -> +JACOBI_FLOOR."""
    f2 = np.asarray(f2, dtype=np.float64)
    mag = np.maximum(np.abs(f2), JACOBI_FLOOR)
    return 1.0 / np.where(f2 < 0, -mag, mag)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (N_PARAMS,)
    return dict(mu=p[OFF_MU:OFF_MU + 6], sigma=p[OFF_SIGMA:OFF_SIGMA + 6],
                W1=p[OFF_W1:OFF_B1].reshape(HIDDEN, N_FEAT), b1=p[OFF_B1:OFF_W2],
                W2=p[OFF_W2:OFF_B2].reshape(HIDDEN, HIDDEN), b2=p[OFF_B2:OFF_W3],
                w3=p[OFF_W3:OFF_B3], b3=p[OFF_B3])


def pack(d):
    out = np.zeros(N_PARAMS)
    out[OFF_MU:OFF_MU + 6] = d["mu"]
    out[OFF_SIGMA:OFF_SIGMA + 6] = d["sigma"]
    out[OFF_W1:OFF_B1] = np.asarray(d["W1"]).ravel()
    out[OFF_B1:OFF_W2] = d["b1"]
    out[OFF_W2:OFF_B2] = np.asarray(d["W2"]).ravel()
    out[OFF_B2:OFF_W3] = d["b2"]
    out[OFF_W3:OFF_B3] = d["w3"]
    out[OFF_B3] = d["b3"]
    return out


def row_abs_sum(H, U=None):
    """(|H| 1)_i of the full symmetric H = U + U^T - D: sum of |h_ij| over the whole row."""
    if U is None:
        U = to_scipy_upper(H)
    A = abs(U)
    d = np.abs(U.diagonal())
    return np.asarray(A.sum(axis=1)).ravel() + np.asarray(A.sum(axis=0)).ravel() - d


def residual(H, X, theta, U=None):
    """R = H X - X diag(theta) (Eq. (rblock)), float64."""
    X = np.asarray(X, dtype=np.float64)
    return sym_upper_matmul(H, X, U) - X * np.asarray(theta, dtype=np.float64)[None, :]


def features(H, theta, R, U=None):
    """F[i, j, :] = (f0..f5) of the module docstring for residual block R (n x m)."""
    if U is None:
        U = to_scipy_upper(H)
    n, m = R.shape
    d = U.diagonal()
    theta = np.asarray(theta, dtype=np.float64)
    HR = sym_upper_matmul(H, R, U)
    nr = np.sqrt((R * R).sum(axis=0))
    scale = np.where(nr > 0, np.sqrt(n) / np.where(nr > 0, nr, 1.0), 0.0)
    F = np.empty((n, m, N_FEAT))
    F[:, :, 0] = d[:, None]
    F[:, :, 1] = theta[None, :]
    F[:, :, 2] = d[:, None] - theta[None, :]
    F[:, :, 3] = row_abs_sum(H, U)[:, None]
    F[:, :, 4] = R * scale[None, :]
    F[:, :, 5] = (HR - d[:, None] * R) * scale[None, :]
    return F


def forward(params, F):
    """m = J(f2) (1 + MLP(standardise(F))) for F (..., 6); returns (m, cache for backward)."""
    P = unpack(params)
    F = np.asarray(F, dtype=np.float64)
    u = (F - P["mu"]) / P["sigma"]
    a1 = u @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ P["w3"] + P["b3"]
    J = jacobi_scale(F[..., 2])
    return J * (1.0 + o), dict(u=u, a1=a1, h1=h1, a2=a2, h2=h2, J=J)


def backward(params, cache, dm):
    """Gradient of sum(dm * m) with respect to the flat parameters (the fixed mu, sigma get
    zero).  dm/do = J, then the chain rule through the two ReLU layers; ReLU'(0) = 0."""
    P = unpack(params)
    u = cache["u"].reshape(-1, N_FEAT)
    a1 = cache["a1"].reshape(-1, HIDDEN)
    h1 = cache["h1"].reshape(-1, HIDDEN)
    a2 = cache["a2"].reshape(-1, HIDDEN)
    h2 = cache["h2"].reshape(-1, HIDDEN)
    g = (np.asarray(dm, dtype=np.float64) * cache["J"]).reshape(-1)
    dw3 = h2.T @ g
    db3 = g.sum()
    da2 = (g[:, None] * P["w3"][None, :]) * (a2 > 0)
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    da1 = (da2 @ P["W2"]) * (a1 > 0)
    dW1 = da1.T @ u
    db1 = da1.sum(axis=0)
    return pack(dict(mu=np.zeros(6), sigma=np.zeros(6), W1=dW1, b1=db1, W2=dW2, b2=db2, w3=dw3, b3=db3))


def correction_target(X, Xstar):
    """z_j = x_j - X* p / (p^T p), p = X*^T x_j (module docstring), and the column weights
    c_j = 1 / ||z_j||^2 (0 where z_j or p vanishes)."""
    X = np.asarray(X, dtype=np.float64)
    Xs = np.asarray(Xstar, dtype=np.float64)
    Pm = Xs.T @ X                       # k x m
    s = (Pm * Pm).sum(axis=0)
    ok = s > 0
    Z = X - Xs @ (Pm / np.where(ok, s, 1.0)[None, :])
    Z[:, ~ok] = 0.0
    zz = (Z * Z).sum(axis=0)
    c = np.where(ok & (zz > 0), 1.0 / np.where(zz > 0, zz, 1.0), 0.0)
    return Z, c


def loss(params, F, R, Z, c):
    """L and dL/dm of the module docstring (c_j = 1/||z_j||^2, or 0 to leave column j out)."""
    m, cache = forward(params, F)
    c = np.asarray(c, dtype=np.float64)
    nJ = max(int((c > 0).sum()), 1)
    err = m * R - Z
    L = float((err * err * c[None, :]).sum() / nJ)
    dm = 2.0 * err * R * c[None, :] / nJ
    return L, dm, cache


def loss_grad(params, F, R, Z, c):
    L, dm, cache = loss(params, F, R, Z, c)
    return L, backward(params, cache, dm)


def apply(params, F, R, diagH, theta, floor=2.0):
    """w = m r, entrywise Jacobi where m r is not finite."""
    m, _ = forward(params, F)
    W = m * np.asarray(R, dtype=np.float64)
    bad = ~np.isfinite(W)
    if bad.any():
        J = jacobi_apply(diagH, theta, R, floor)
        W[bad] = J[bad]
    return W


def adam_step(params, grad, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of the trained entries (index >= 12); returns the new
    (params, m1, m2).  t is the 1-based step number of the bias corrections."""
    p = np.array(params, dtype=np.float64)
    g = np.asarray(grad, dtype=np.float64)
    m1 = beta1 * np.asarray(m1) + (1 - beta1) * g
    m2 = beta2 * np.asarray(m2) + (1 - beta2) * g * g
    mh = m1 / (1 - beta1 ** t)
    vh = m2 / (1 - beta2 ** t)
    upd = lr * mh / (np.sqrt(vh) + eps)
    p[N_FIXED:] -= upd[N_FIXED:]
    m1[:N_FIXED] = 0.0
    m2[:N_FIXED] = 0.0
    return p, m1, m2


def feature_stats(Fs):
    """mu, sigma of the features over a list of (n, m, 6) arrays (sigma floored at 1e-6)."""
    A = np.concatenate([np.asarray(F).reshape(-1, N_FEAT) for F in Fs])
    mu = A.mean(axis=0)
    sg = np.maximum(A.std(axis=0), 1e-6)
    return mu, sg
