"""GPU parity of the dense steps around the SpMM, through the C ABI: Gram products, CholQR2,
the projected eigensolver, the LOBPCG Rayleigh-Ritz pencil, the RMM-DIIS 2x2 Rayleigh-Ritz and
the DIIS least squares -- each against the FP64 oracle on the same inputs."""
import numpy as np
import pytest

import oracle as O
from gen import laplacian_kron, laplacian_kron_eigs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def B():
    from paper_2305_15552_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("n,nb", [(1, 4), (31, 8), (5000 + 17, 16), (100003, 8), (4096, 48)])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_gram(n, nb, dt):
    rng = np.random.default_rng(n + nb)
    A = torch.tensor(rng.standard_normal((n, nb)), dtype=dt, device="cuda")
    Bm = torch.tensor(rng.standard_normal((n, nb)), dtype=dt, device="cuda")
    G = B().gram(A, Bm).cpu().numpy()
    Ae, Be = A.double().cpu().numpy(), Bm.double().cpu().numpy()
    ref = O.gram(Ae, Be)
    bound = np.abs(Ae).T @ np.abs(Be)
    # FP32: products rounded once (2^-24) + 32-term FP32 partial sums; FP64: n * 2^-53
    tol = (2.0 ** -24 * 40 if dt == torch.float32 else 2.0 ** -53 * (n + 10)) * bound + 1e-300
    assert np.all(np.abs(G - ref) <= tol)
    G2 = B().gram(A, Bm).cpu().numpy()
    assert np.array_equal(G, G2)


@pytest.mark.parametrize("k", [1, 6, 16, 48])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_cholqr2(k, dt):
    n = 20000 + 3
    rng = np.random.default_rng(k)
    X = rng.standard_normal((n, k))
    X[:, -1] += 0.5 * X[:, 0]
    Xt = torch.tensor(X, dtype=dt, device="cuda")
    Xe = Xt.double().cpu().numpy()
    Q, R = B().cholqr2(Xt)
    Q, R = Q.double().cpu().numpy(), R.cpu().numpy()
    eps = 2.0 ** -24 if dt == torch.float32 else 2.0 ** -53
    assert np.abs(Q.T @ Q - np.eye(k)).max() < 200 * eps * np.sqrt(k) * 10
    assert np.abs(Q @ R - Xe).max() < 1e3 * eps * np.abs(Xe).max()
    Qr, Rr = O.cholqr2(Xe)
    np.testing.assert_allclose(R, Rr, rtol=0, atol=1e3 * eps * np.abs(Rr).max())


def test_cholqr2_breakdown():
    from paper_2305_15552_gb300 import binding
    X = np.random.default_rng(0).standard_normal((1000, 4))
    X[:, 3] = X[:, 1]
    with pytest.raises(binding.EigError) as e:
        B().cholqr2(torch.tensor(X, device="cuda"))
    assert e.value.status == binding.EIG_EBREAKDOWN


def _sym(k, seed, kind):
    rng = np.random.default_rng(seed)
    if kind == "random":
        A = rng.standard_normal((k, k))
        return A + A.T
    if kind == "degenerate":                      # exact multiplicities
        d = np.repeat(np.arange(k // 3 + 1, dtype=float), 3)[:k]
        Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
        return (Q * d) @ Q.T
    if kind == "graded":                          # eigenvalues over 12 decades
        d = np.logspace(-6, 6, k)
        Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
        return (Q * d) @ Q.T
    if kind == "laplacian":
        return O.to_dense(laplacian_kron([3, 4, 4]))[:k, :k]


@pytest.mark.parametrize("k,m", [(1, 1), (2, 1), (8, 8), (24, 8), (48, 16), (48, 48), (130, 16), (400, 32)])
@pytest.mark.parametrize("kind", ["random", "degenerate", "graded", "laplacian"])
def test_small_syev(k, m, kind):
    if kind == "laplacian" and k > 48:
        pytest.skip("laplacian fixture has 48 rows")
    A = _sym(k, k * 7 + m, kind)
    w, Z = B().small_syev(torch.tensor(A, device="cuda"), m)
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    wr = np.linalg.eigvalsh(A)[:m]
    scale = max(np.abs(np.linalg.eigvalsh(A)).max(), 1e-300)
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-12 * scale)
    assert np.abs(Z.T @ Z - np.eye(m)).max() < 1e-10
    res = np.linalg.norm(A @ Z - Z * w, axis=0)
    assert res.max() <= 1e-10 * scale


def test_small_syev_laplacian_closed_form():
    H = laplacian_kron([4, 5, 6])
    A = O.to_dense(H)
    w, _ = B().small_syev(torch.tensor(A, device="cuda"), 20)
    np.testing.assert_allclose(w.cpu().numpy(), laplacian_kron_eigs([4, 5, 6])[:20], atol=1e-12)


@pytest.mark.parametrize("k,nb", [(16, 16), (32, 16), (48, 16), (24, 8)])
def test_small_rr_matches_oracle_pencil(k, nb):
    rng = np.random.default_rng(k + nb)
    S = rng.standard_normal((300, k))
    S[:, k // 2:] *= 1e-3                         # small W/P columns as near convergence
    Hm = O.to_dense(laplacian_kron([6, 7, 8]))[:300, :300]
    A, G = S.T @ Hm @ S, S.T @ S
    th, C, info = B().small_rr(torch.tensor(A, device="cuda"), torch.tensor(G, device="cuda"), nb)
    assert info == 0
    th, C = th.cpu().numpy(), C.cpu().numpy()
    thr, Cr = O.rayleigh_ritz_projected(A, G, nb)
    np.testing.assert_allclose(th, thr, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(C.T @ G @ C, np.eye(nb), atol=1e-9)
    # same Ritz vectors up to sign (simple eigenvalues here)
    X, Xr = S @ C, S @ Cr
    assert np.all(np.abs(np.abs(np.sum(X * Xr, axis=0)) - 1) < 1e-8)


def test_small_rr_breakdown_flag():
    S = np.random.default_rng(1).standard_normal((100, 8))
    S[:, 7] = S[:, 6]
    Hm = np.diag(np.arange(100.0))
    _, _, info = B().small_rr(torch.tensor(S.T @ Hm @ S, device="cuda"), torch.tensor(S.T @ S, device="cuda"), 4)
    assert info == 1


def test_rmm_rr2_matches_oracle():
    rng = np.random.default_rng(3)
    m = 8
    M = rng.standard_normal((60, 60)); M = M + M.T
    dots = np.zeros((m, 6))
    ref = []
    for j in range(m):
        x, r = rng.standard_normal(60), rng.standard_normal(60) * 10.0 ** -(j % 4)
        Hx, Hr = M @ x, M @ r
        dots[j] = [x @ x, x @ Hx, x @ r, r @ r, x @ Hr, r @ Hr]
        ref.append(O.rr2(x, r, Hx, Hr))
    act = torch.ones(m, dtype=torch.int32, device="cuda")
    th, g = B().rmm_rr2(torch.tensor(dots, device="cuda"), act)
    th, g = th.cpu().numpy(), g.cpu().numpy()
    for j in range(m):
        np.testing.assert_allclose(th[j], ref[j][0], rtol=1e-10)
        gr = ref[j][1]
        assert g[j][0] <= 0 and gr[0] <= 0
        np.testing.assert_allclose(g[j], gr, rtol=1e-7, atol=1e-12 * np.abs(gr).max())
    act[3] = 0
    th, g = B().rmm_rr2(torch.tensor(dots, device="cuda"), act)
    assert g[3, 1].item() == 0.0


@pytest.mark.parametrize("s", [1, 2, 5, 10, 20])
def test_rmm_diis_matches_oracle(s):
    rng = np.random.default_rng(s)
    m = 4
    Bm = np.zeros((m, 20, 20))
    slots = [(3 + i) % 20 for i in range(s)]           # a wrapped ring-buffer window
    rs = [[rng.standard_normal(200) * 0.5 ** i for i in range(s)] for _ in range(m)]
    for j in range(m):
        for a in range(s):
            for b in range(s):
                Bm[j, slots[a], slots[b]] = rs[j][a] @ rs[j][b]
    act = torch.ones(m, dtype=torch.int32, device="cuda")
    al = B().rmm_diis(torch.tensor(Bm, device="cuda"), slots, act).cpu().numpy()
    for j in range(m):
        ref = O.diis_coefficients(rs[j])
        np.testing.assert_allclose(al[j, :s], ref, rtol=1e-8, atol=1e-10)
        assert abs(al[j, :s].sum() - 1) < 1e-12
