"""Learned per-row preconditioner on the GPU against the FP64 oracle (oracle/learned.py):
samples (features, residuals, targets, column weights), the network forward, the fused loss
gradient, the Adam step and the preconditioner apply, all through the C ABI; then the solver
with the learned K (convergence to the oracle's eigenvalues, Jacobi fallback), and training on
a small matrix family (the trained network predicts the correction better than Jacobi)."""
import numpy as np
import pytest

import oracle as O
from oracle import learned as L
from gen import ci_matrix, random_block, family_perturbation, family_member, principal_submatrix, pad_rows

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, NNZ, NEV, NB, K = 6003, 120, 8, 8, 8     # n * m = 48024 entries: 375 tiles of 128 + a ragged 24


@pytest.fixture(scope="module")
def H():
    return ci_matrix(N, NNZ, 64, seed=2, storage="f64")


@pytest.fixture(scope="module")
def solver(H):
    from paper_2305_15552_gb300.binding import Solver
    S = Solver(H, NEV, NB)
    yield S
    S.close()


@pytest.fixture(scope="module")
def H32():
    """The same matrix with FP32 values (the SpMM of FP32 vectors takes FP32 or BF16 values)."""
    return ci_matrix(N, NNZ, 64, seed=2, storage="f32")


@pytest.fixture(scope="module")
def solver32(H32):
    from paper_2305_15552_gb300.binding import Solver
    S = Solver(H32, NEV, NB)
    yield S
    S.close()


@pytest.fixture(scope="module")
def pairs(H):
    """Approximate Ritz pairs (a few oracle LOBPCG steps) and an orthonormal X* of the wanted space."""
    U = O.to_scipy_upper(H)
    rng = np.random.default_rng(4)
    X0 = random_block(N, NB, seed=5)
    res = O.lobpcg(H, X0, NEV, tol=1e-9, maxiter=200)
    Xstar = np.linalg.qr(res.X[:, :K])[0]
    # perturbed iterate: X* plus noise, orthonormalised, Rayleigh quotients as theta
    X = Xstar + 1e-2 * rng.standard_normal((N, NEV))
    X = np.linalg.qr(X)[0]
    th = np.einsum("ij,ij->j", X, O.sym_upper_matmul(H, X, U))
    return X, th, Xstar, U


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def test_sample_matches_oracle(H, solver, pairs):
    X, th, Xstar, U = pairs
    s = solver.lp_sample(_dev(X), th, _dev(Xstar), target=0)
    R = L.residual(H, X, th, U)
    F = L.features(H, th, R, U).reshape(-1, 6)
    Fg = s["F"].cpu().numpy().astype(np.float64)
    for q in range(6):
        scale = max(np.abs(F[:, q]).max(), 1e-30)
        np.testing.assert_allclose(Fg[:, q], F[:, q], rtol=0, atol=2e-7 * scale, err_msg=f"feature {q}")
    np.testing.assert_allclose(s["r"].cpu().numpy(), R.ravel(), rtol=0, atol=2e-7 * np.abs(R).max())
    Z, c = L.correction_target(X, Xstar)
    np.testing.assert_allclose(s["z"].cpu().numpy(), Z.ravel(), rtol=0, atol=2e-7 * np.abs(Z).max())
    nJ = int((c > 0).sum())
    np.testing.assert_allclose(s["colw"].cpu().numpy(), c / nJ, rtol=1e-10, atol=0)
    # the absolute row sums (fixed-point accumulation on the GPU)
    np.testing.assert_allclose(Fg.reshape(N, NEV, 6)[:, 0, 3], L.row_abs_sum(H, U), rtol=1e-7)


def test_jacobi_target_sample(H, solver, pairs):
    X, th, _, U = pairs
    s = solver.lp_sample(_dev(X), th, None, target=1, floor=2.0)
    R = L.residual(H, X, th, U)
    Zj = O.jacobi_apply(H.diagonal_f64(), th, R, 2.0)
    np.testing.assert_allclose(s["z"].cpu().numpy(), Zj.ravel(), rtol=0, atol=2e-7 * np.abs(Zj).max())
    zz = (Zj * Zj).sum(axis=0)
    np.testing.assert_allclose(s["colw"].cpu().numpy(), 1.0 / (NEV * zz), rtol=1e-10)


def _params(seed=1, scale=0.4):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(L.N_PARAMS) * scale
    p[0:6] = rng.standard_normal(6) * 0.1
    p[6:12] = 0.5 + rng.random(6)
    return p.astype(np.float32)


def _standardised_params(sample, seed=1):
    from paper_2305_15552_gb300 import learned as LG
    mu, sg = LG.feature_stats([sample])
    p = LG.init_params(mu, sg, seed=seed)
    return p


def test_forward_matches_oracle(solver, pairs):
    from paper_2305_15552_gb300 import binding as B
    X, th, Xstar, _ = pairs
    s = solver.lp_sample(_dev(X), th, _dev(Xstar))
    p = _standardised_params(s)
    m = B.lp_forward(p, s["F"]).cpu().numpy()
    mo, _ = L.forward(p.astype(np.float64), s["F"].cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(m, mo, rtol=0, atol=2e-5 * max(1.0, np.abs(mo).max()))


def test_grad_matches_oracle_and_is_deterministic(solver, pairs):
    from paper_2305_15552_gb300 import binding as B
    X, th, Xstar, _ = pairs
    s = solver.lp_sample(_dev(X), th, _dev(Xstar))
    p = _standardised_params(s, seed=3)
    g = B.lp_grad(_dev(p), s).cpu().numpy()
    g2 = B.lp_grad(_dev(p), s).cpu().numpy()
    assert np.array_equal(g, g2), "gradient not deterministic"
    colw = s["colw"].cpu().numpy()
    nJ = int((colw > 0).sum())
    Lo, go = L.loss_grad(p.astype(np.float64), s["F"].cpu().numpy().astype(np.float64).reshape(N, NEV, 6),
                         s["r"].cpu().numpy().astype(np.float64).reshape(N, NEV),
                         s["z"].cpu().numpy().astype(np.float64).reshape(N, NEV), colw * nJ)
    assert g[-1] == pytest.approx(Lo, rel=1e-5)
    gt = go[L.N_FIXED:]
    assert np.linalg.norm(g[:-1] - gt) <= 1e-4 * np.linalg.norm(gt)
    # blocks separately (a transposed or misplaced block would pass a global norm only by luck)
    for a, b in [(12, 204), (204, 236), (236, 1260), (1260, 1292), (1292, 1324), (1324, 1325)]:
        ga, gb = g[a - 12:b - 12], gt[a - 12:b - 12]
        assert np.linalg.norm(ga - gb) <= 1e-4 * max(np.linalg.norm(gb), 1e-3 * np.linalg.norm(gt)), (a, b)


def test_adam_matches_oracle():
    from paper_2305_15552_gb300 import binding as B
    rng = np.random.default_rng(9)
    p = rng.standard_normal(L.N_PARAMS).astype(np.float32)
    pd, m1, m2 = _dev(p), torch.zeros(L.N_PARAMS, device="cuda"), torch.zeros(L.N_PARAMS, device="cuda")
    po, mo1, mo2 = p.astype(np.float64), np.zeros(L.N_PARAMS), np.zeros(L.N_PARAMS)
    for t in (1, 2, 3):
        g = rng.standard_normal(L.N_PARAMS)
        gd = _dev(g[L.N_FIXED:].copy())
        B.lp_adam(pd, gd, m1, m2, t, 1e-2)
        po, mo1, mo2 = L.adam_step(po, g, mo1, mo2, t, 1e-2)
    np.testing.assert_allclose(pd.cpu().numpy(), po, rtol=1e-6, atol=1e-6)
    assert np.array_equal(pd.cpu().numpy()[:12], p[:12])


@pytest.mark.parametrize("vt", ["f64", "f32"])
def test_apply_matches_oracle(H, solver, H32, solver32, pairs, vt):
    X, th, Xstar, U = pairs
    s = solver.lp_sample(_dev(X), th, _dev(Xstar))
    if vt == "f32":
        H, solver, U = H32, solver32, O.to_scipy_upper(H32)
    p = _standardised_params(s, seed=5)
    R = L.residual(H, X, th, U)
    dt = torch.float64 if vt == "f64" else torch.float32
    W = solver.lp_apply(p, _dev(R).to(dt), th).cpu().numpy().astype(np.float64)
    Rin = R if vt == "f64" else R.astype(np.float32).astype(np.float64)
    Wo = L.apply(p.astype(np.float64), L.features(H, th, Rin, U), Rin, H.diagonal_f64(), th)
    tol = 5e-5 if vt == "f64" else 2e-4
    np.testing.assert_allclose(W, Wo, rtol=0, atol=tol * np.abs(Wo).max())
    # a broken network falls back to Jacobi entrywise
    pn = p.copy()
    pn[L.OFF_B3] = np.nan
    Wn = solver.lp_apply(pn, _dev(R).to(dt), th).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(Wn, O.jacobi_apply(H.diagonal_f64(), th, Rin), rtol=1e-6 if vt == "f32" else 1e-15,
                               atol=0)


def test_lobpcg_zero_output_layer_is_jacobi(solver):
    """o = 0 (zero output layer) makes m the Jacobi scale: the solve follows precond = 1 (the scale
    is rounded differently from the update kernel's division, so LOBPCG's iteration count, which
    is sensitive to rounding, may differ by up to a quarter)."""
    p = _params(seed=2)
    p[L.OFF_W3:L.OFF_B3 + 1] = 0.0
    X0 = random_block(N, NB, seed=11)
    rcj, stj = solver.solve("lobpcg", X0=X0, vec_type="f64", tol=1e-7, maxiter=400, precond=1)
    thj = solver.ritz()[0]
    rc, st = solver.solve("lobpcg", X0=X0, vec_type="f64", tol=1e-7, maxiter=400, precond=2, lp_params=p)
    th = solver.ritz()[0]
    assert rc == rcj and abs(st["iterations_front"] - stj["iterations_front"]) <= max(2, stj["iterations_front"] // 4)
    np.testing.assert_allclose(th, thj, rtol=1e-9)
    assert st["lp_spmm_calls"] == st["iterations_front"] + 1 and st["precond_fallback"] == 0


def test_lobpcg_nan_network_falls_back_to_jacobi(H, solver):
    """A network whose output is NaN: every entry takes the Jacobi value, the solve switches to
    Jacobi after its first step and then runs as precond = 1 does."""
    p = np.zeros(L.N_PARAMS, dtype=np.float32)
    p[6:12] = 1.0
    p[L.OFF_B3] = np.nan
    X0 = random_block(N, NB, seed=11)
    rcj, stj = solver.solve("lobpcg", X0=X0, vec_type="f64", tol=1e-7, maxiter=400, precond=1)
    thj = solver.ritz()[0]
    rc, st = solver.solve("lobpcg", X0=X0, vec_type="f64", tol=1e-7, maxiter=400, precond=2, lp_params=p)
    th, _, rel = solver.ritz()
    print(f"Jacobi: rc {rcj}, {stj['iterations_front']} iterations; NaN network: rc {rc}, "
          f"{st['iterations_front']} iterations, fallback {st['precond_fallback']}")
    assert (st["precond_fallback"] & 0xFFFF) == 1
    assert rc == rcj and abs(st["iterations_front"] - stj["iterations_front"]) <= 2
    np.testing.assert_allclose(th, thj, rtol=1e-9)
    if rc == 0:
        ref = O.lobpcg(H, X0, NEV, tol=1e-9, maxiter=300)
        np.testing.assert_allclose(th, np.sort(ref.theta[:NEV]), rtol=1e-7)


def _small_space_start(H, n0):
    """Zero-padded lowest eigenvectors of the leading n0 x n0 block (GPU solve at 1e-4)."""
    from paper_2305_15552_gb300.binding import Solver
    S0 = Solver(principal_submatrix(H, n0), NB, NB)
    S0.solve("hybrid", vec_type="f32", tol=1e-4)
    _, Z0, _ = S0.ritz()
    S0.close()
    return pad_rows(Z0, H.n)


@pytest.fixture(scope="module")
def family():
    """H(g) = H0 + g V (n = 20000, ~150 nnz/row, FP32 values), g uniform in [0.5, 1.5]: samples
    of 6 training and 2 held-out members along LOBPCG from the small-space start, and a network
    trained on the training samples."""
    from paper_2305_15552_gb300.binding import Solver
    from paper_2305_15552_gb300 import learned as LG
    n = 20000
    H0 = ci_matrix(n, 150, 64, seed=7, storage="f32")
    V = family_perturbation(H0, seed=8)
    gs = np.random.default_rng(3).uniform(0.5, 1.5, 8)
    train_s, held_s, starts = [], [], []
    for q, g in enumerate(gs):
        Hq = family_member(H0, V, g)
        X0 = _small_space_start(Hq, n // 10)
        starts.append(X0)
        S = Solver(Hq, NEV, NB)
        smp = LG.collect_samples(S, X0, iters=(0, 1, 2, 3, 4, 6, 8, 11))
        (train_s if q < 6 else held_s).extend(smp)
        S.close()
    p0 = LG.init_params(*LG.feature_stats(train_s), seed=0)
    p, hist = LG.train(train_s, p0, epochs=40, lr=1e-3)
    return dict(H0=H0, V=V, gs=gs, starts=starts, train=train_s, held=held_s, p0=p0, p=p, hist=hist)


def test_training_beats_jacobi_on_held_out_family(family):
    """After training on the correction targets, the network's loss on held-out samples is below
    the Jacobi K's."""
    from paper_2305_15552_gb300 import learned as LG
    assert len(family["train"]) >= 6 and len(family["held"]) >= 2
    hist = family["hist"]
    assert hist[-1] < hist[0]
    learned = LG.mean_loss(family["held"], family["p"])
    start = LG.mean_loss(family["held"], family["p0"])
    jac = float(np.mean([LG.jacobi_loss(s) for s in family["held"]]))
    print(f"held-out loss: learned {learned:.4f}, Jacobi {jac:.4f}, untrained (= Jacobi scale) {start:.4f}; "
          f"training loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    assert start == pytest.approx(jac, rel=1e-4)
    assert learned < jac


def test_hybrid_with_trained_k_fp32(family):
    """The hybrid (LOBPCG front, RMM-DIIS) with the trained K on a held-out member converges to
    the oracle's eigenvalues at relative residual 1e-6."""
    from paper_2305_15552_gb300.binding import Solver
    H = family_member(family["H0"], family["V"], family["gs"][7])
    X0 = family["starts"][7]
    S = Solver(H, NEV, NB)
    opts = dict(vec_type="f32", switch_res=1e-2, switch_tau=0.0, maxiter=300)
    rcj, stj = S.solve("hybrid", X0=X0, precond=1, rmm_precond=1, **opts)
    rc, st = S.solve("hybrid", X0=X0, precond=2, rmm_precond=2, lp_params=family["p"], **opts)
    th, Xg, rel = S.ritz()
    S.close()
    print(f"hybrid, held-out member: Jacobi {stj['iterations_front']}+{stj['iterations_rmm']} iterations "
          f"({stj['spmm_calls']} SpMM), learned {st['iterations_front']}+{st['iterations_rmm']} iterations "
          f"({st['spmm_calls']} SpMM, {st['lp_spmm_calls']} for features, K fallback {st['precond_fallback']:#x}, "
          f"LOBPCG safety net {st['iterations_fallback']} (Jacobi run: {stj['iterations_fallback']})")
    assert rc == 0 and np.all(rel <= 1e-6)
    assert np.all(O.true_relres(H, th, Xg) <= 1.05e-6)
    ref = O.lobpcg(H, X0, NEV, tol=1e-9, maxiter=400)
    np.testing.assert_allclose(th, np.sort(ref.theta[:NEV]), rtol=1e-6)
