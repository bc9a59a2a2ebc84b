"""FP64 CPU oracle for the hybrid eigensolver hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct restatements of what the paper computes, in float64
with numpy/scipy primitives (sparse matmul, dense eigh, Cholesky, triangular solve).
Every function cites the passage it follows.  Only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline/reference leg may import this package; the product
(paper_2305_15552_gb300) never imports or calls it, and it imports nothing from the
product.  The two share only the seeded input generators in gen/.

Layers
  * exact definitions: sym_upper_matmul (Y = H X for half-stored H), dense lowest
    eigenpairs (numpy eigh), Gram, CholQR2, Rayleigh-Ritz;
  * the paper's algorithms step by step: Lanczos (Sec. 2.1), block Lanczos (Alg. 1),
    LOBPCG (Alg. 2), ChebFSI (Alg. 3), RMM-DIIS (Alg. 4), hybrids (Sec. 4);
  * certification helpers (true residuals, residual/Kato-Temple bounds);
  * the learned per-row preconditioner (oracle.learned): features, MLP forward/backward,
    correction targets, loss and Adam step, in float64.

Parity pins: every function is checked in tests/test_oracle_*.py against closed
forms (Kronecker-sum Laplacian spectra, Chebyshev T_m(cos t) = cos(m t), 2x2 pencil
roots, two-vector DIIS), brute-force dense diagonalisation and invariants.
"""
from .spmm import sym_upper_matmul, to_scipy_upper, to_dense, spmv_count_per_spmm, parallel_upper, ParallelUpper
from .dense import lowest_eigpairs, eigh_sorted
from .blocks import gram, cholqr, cholqr2, rayleigh_ritz, rayleigh_ritz_projected, orthonormal_basis
from .precond import jacobi_apply
from .lanczos import lanczos
from .block_lanczos import block_lanczos, thick_restart
from .lobpcg import lobpcg
from .chebfsi import chebfsi, lambda_ub_estimate, cheb_filter
from .rmmdiis import rmmdiis, diis_coefficients, diis_extrapolate, rr2
from .hybrid import hybrid, switch_tau, gap_condition
from .certify import true_relres, residual_bound, kato_temple, missed_eigenvalues

__all__ = [n for n in dir() if not n.startswith("_")]
