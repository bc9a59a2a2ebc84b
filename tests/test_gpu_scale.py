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
  20,000-row block (Cauchy interlacing), which interior eigenpairs would not;
* at 8M, a second GPU method (LOBPCG with FP64 vectors, no RMM-DIIS) from the same start returns
  the same ten values to 1e-9 relative (a cross-check of two GPU methods, not of the oracle: the
  oracle cannot solve 8M rows within a test);
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
def start(H8M):
    """Zero-padded lowest eigenvectors of the leading n/10 principal block (GPU LOBPCG with FP64
    vectors to relative residual 1e-6 or 2000 iterations, from a seeded random block: a start,
    not a result)."""
    from paper_2305_15552_gb300.binding import Solver
    n0 = N // 10
    S0 = Solver(principal_submatrix(H8M, n0), NB, NB)
    rc, st = S0.solve("lobpcg", vec_type="f64", tol=1e-6, maxiter=2000, seed=1)
    _, Z0, rel0 = S0.ritz()
    assert np.all(np.isfinite(Z0)) and np.max(rel0[:NEV]) < 1e-3, (rc, st, rel0)
    S0.close()
    return pad_rows(Z0, N)


def interlacing_bound(H, m, k):
    """The oracle's lowest k eigenvalues of the leading m x m principal block: by Cauchy
    interlacing lambda_j(H) <= lambda_j(H_m), so a result above them is not the lowest pairs."""
    Hm = principal_submatrix(H, m)
    X = np.random.default_rng(5).standard_normal((m, 2 * k))
    r = O.lobpcg(Hm, X, k, tol=1e-9, maxiter=500)
    assert r.converged
    return np.sort(r.theta[:k])


def test_hybrid_8M_fp32_certified_by_oracle(H8M, start):
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
    # the lowest pairs, not interior ones: below the oracle's eigenvalues of a leading block
    assert np.all(th <= interlacing_bound(H, 20000, NEV) + 1e-9), th
    U = O.to_scipy_upper(H)
    tr = O.true_relres(H, th, X, U)
    assert np.all(tr <= 1.05e-6), tr
    np.testing.assert_allclose(rel, tr, rtol=1e-2, atol=1e-9)
    # the same ten eigenvalues from LOBPCG with FP64 vectors (no RMM-DIIS) from the same start
    S2 = Solver(H, NEV, NB)
    rc2, st2 = S2.solve("lobpcg", X0=start, vec_type="f64", tol=1e-7, maxiter=400)
    assert rc2 == 0, st2
    th2, X2, _ = S2.ritz()
    S2.close()
    np.testing.assert_allclose(th, th2, rtol=1e-9, atol=0)
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
