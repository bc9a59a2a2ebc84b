"""Mixed precision at scale: 8,000,000 rows, ~500 nnz/row (2.0e9 stored nonzeros, int64 row
pointers, int32 columns), FP32 values and vectors, n_ev = 10, block 16 -- the hybrid solve of the
paper (LOBPCG front to relative residual 1e-2 and the gap condition, preconditioned RMM-DIIS to
1e-6) on the GPU.

Checks, all against FP64 arithmetic outside the CUDA path:
* the oracle's own FP64 product of the full matrix gives the true residual of every returned pair:
  it must be <= 1e-6 and agree with the library's certified value;
* residual bound: some eigenvalue of H lies within ||r|| of each theta, so |dlambda|/|lambda| <=
  relres <= 1e-6 for the pair it certifies;
* the lowest pairs: every theta_j lies at or below the oracle's j-th eigenvalue of the leading
  20,000-row block (Cauchy interlacing), which interior eigenpairs would not (the start comes
  from that block through the n/10 block, the smaller-model-space start of Sec. 3.1);
* at 8M, a second GPU method (LOBPCG with FP64 vectors, no RMM-DIIS) from the same start returns
  the same ten values within the two results' residual bounds (a cross-check of two GPU methods,
  not of the oracle: the oracle cannot solve 8M rows within a test);
* which eigenvalues, against the oracle: at 200,000 rows of the same generator and density the
  hybrid's ten eigenvalues match the oracle's FP64 LOBPCG to 1e-6 relative, and Lanczos from a
  random start (the oracle's missed-eigenvalue guard) finds none below them that they lack.
At 8M the wanted ten include a whole near-degenerate shell, on which RMM-DIIS alone can leave one
or two vectors unconverged or collapsed together; the hybrid then finishes with LOBPCG on FP64
vectors from the RMM-DIIS result (the library's fallback, reported in iterations_fallback).
The matrix generation alone takes about a minute on the host."""
import numpy as np
import pytest

import oracle as O
from gen import ci_matrix, principal_submatrix, pad_rows

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, NNZ_ROW, NEV, NB = 8_000_000, 500, 10, 16


@pytest.fixture(scope="module")
def H8M():
    return ci_matrix(N, NNZ_ROW, 256, seed=1, storage="f32")


@pytest.fixture(scope="module")
def block20k(H8M):
    """The oracle's lowest eigenpairs of the leading 20,000-row block (LOBPCG from a seeded
    random block, FP64, relative residual 1e-9)."""
    m = 20000
    Hm = principal_submatrix(H8M, m)
    X = np.random.default_rng(5).standard_normal((m, 2 * NB))
    r = O.lobpcg(Hm, X, NB, tol=1e-9, maxiter=500)
    assert r.converged
    order = np.argsort(r.theta)
    return r.theta[order], r.X[:, order]


@pytest.fixture(scope="module")
def start(H8M, block20k):
    """The smaller-model-space start of Sec. 3.1, in two stages: the oracle's 20,000-row block
    eigenvectors, zero-padded, start GPU LOBPCG (FP64 vectors, relative residual 1e-6) on the
    leading n/10 block, whose Ritz vectors, zero-padded, start the 8M solve.  (From a random
    block, the shifted Jacobi preconditioner can pull LOBPCG onto a cluster of the interior of
    this spectrum at n/10 rows: the lowest pairs are localised in the first rows, where a random
    block has little weight.)"""
    from paper_2305_15552_gb300.binding import Solver
    n0 = N // 10
    th20, X20 = block20k
    S0 = Solver(principal_submatrix(H8M, n0), NB, NB)
    rc, st = S0.solve("lobpcg", X0=pad_rows(X20[:, :NB], n0), vec_type="f64", tol=1e-6, maxiter=2000)
    th0, Z0, rel0 = S0.ritz()
    S0.close()
    assert np.all(np.isfinite(Z0)) and np.max(rel0[:NEV]) < 1e-3, (rc, st, rel0)
    # Cauchy interlacing: the block's lowest pairs lie at or below the 20,000-row block's
    assert np.all(th0[:NEV] <= th20[:NEV] + 1e-9), (th0, th20)
    return pad_rows(Z0, N)


def test_hybrid_8M_fp32_certified_by_oracle(H8M, start, block20k):
    from paper_2305_15552_gb300.binding import Solver
    H = H8M
    assert H.nnz > 1.9e9 and H.rowptr.dtype == np.int64
    S = Solver(H, NEV, NB)
    info = S.spmm_info()
    rc, st = S.solve("hybrid", X0=start, vec_type="f32", switch_res=1e-2, switch_tau=0.0, switch_gap=0.03,
                     rmm_precond=1, s_max=10, maxiter=500, rmm_maxiter=100)
    assert rc == 0, st
    th, X, rel = S.ritz()
    S.close()
    assert np.all(np.diff(th) >= 0)
    # the lowest pairs, not interior ones: by Cauchy interlacing at or below the oracle's
    # eigenvalues of the leading 20,000-row block
    assert np.all(th <= block20k[0][:NEV] + 1e-9), th
    U = O.to_scipy_upper(H)
    tr = O.true_relres(H, th, X, U)
    assert np.all(tr <= 1.05e-6), tr
    np.testing.assert_allclose(rel, tr, rtol=1e-2, atol=1e-9)
    # the same ten eigenvalues from LOBPCG with FP64 vectors (no RMM-DIIS) from the same start:
    # each theta_j is within ||r_j|| of an eigenvalue, so two results for the same eigenvalue
    # differ by at most the sum of their residual norms
    S2 = Solver(H, NEV, NB)
    rc2, st2 = S2.solve("lobpcg", X0=start, vec_type="f64", tol=1e-7, maxiter=400)
    assert rc2 == 0, st2
    th2, X2, rel2 = S2.ritz()
    S2.close()
    bound = tr * np.abs(th) + rel2 * np.abs(th2) + 1e-12 * np.abs(th2)
    assert np.all(np.abs(th - th2) <= bound), (th, th2, np.abs(th - th2), bound)
    print(f"8M: layout {info['layout']} ({info['device_bytes'] / 1e9:.1f} GB), hybrid {st['iterations_front']} "
          f"LOBPCG + {st['iterations_rmm']} RMM-DIIS + {st['iterations_fallback']} fallback LOBPCG iterations, "
          f"max relres {tr.max():.2e}, theta {th}")


def test_hybrid_200k_eigenvalues_match_oracle():
    """The same generator and density at 200,000 rows, where the oracle finishes: the GPU hybrid
    (FP32 values and vectors) against the oracle's FP64 LOBPCG from the same start, and the
    oracle's missed-eigenvalue guard (Lanczos from one seeded random start) on the GPU result."""
    import os
    from paper_2305_15552_gb300.binding import Solver
    H = ci_matrix(200_000, NNZ_ROW, 256, seed=1, storage="f32")
    n0 = H.n // 10
    S0 = Solver(principal_submatrix(H, n0), NB, NB)
    S0.solve("lobpcg", vec_type="f64", tol=1e-8, maxiter=1000, seed=1)
    _, Z0, _ = S0.ritz()
    S0.close()
    X0 = pad_rows(Z0, H.n)
    S = Solver(H, NEV, NB)
    rc, st = S.solve("hybrid", X0=X0, vec_type="f32", switch_res=1e-2, switch_tau=0.0, switch_gap=0.03,
                     rmm_precond=1, s_max=10, maxiter=500)
    assert rc == 0, st
    assert st["iterations_fallback"] == 0, st
    th, X, rel = S.ritz()
    S.close()
    U = O.parallel_upper(H, os.cpu_count() or 1)
    tr = O.true_relres(H, th, X, U)
    assert np.all(tr <= 1.05e-6), tr
    ref = O.lobpcg(H, X0, NEV, tol=1e-9, maxiter=500, U=U)
    assert ref.converged
    np.testing.assert_allclose(th, ref.theta[:NEV], rtol=1e-6, atol=0)
    assert O.missed_eigenvalues(H, th, NEV, starts=1, U=U).size == 0
    print(f"200k: hybrid {st['iterations_front']} LOBPCG + {st['iterations_rmm']} RMM-DIIS + "
          f"{st['iterations_fallback']} fallback iterations; oracle LOBPCG {ref.iterations} iterations")
