// Small dense kernels, FP64 in and out, double-float inside (projected problems of the Rayleigh-Ritz procedure, Cholesky of
// Gram matrices, DIIS least squares, 2x2 pencils).  Internal interface.
#pragma once
#include "common.cuh"

namespace eig {

// Largest projected dimension the single-CTA solver keeps in shared memory.
constexpr int kSmallSmemMax = 64;
// Largest projected dimension supported at all (global-memory path).
constexpr int kSmallMax = 1024;

// info codes written by the small kernels
enum : int { SMALL_OK = 0, SMALL_BREAKDOWN = 1, SMALL_BAD = 2 };

// Lowest m eigenpairs of the symmetric k x k A (row-major, device), FP64.
// w[m] ascending, Z (k x m, row-major) orthonormal.  work: device scratch of
// small_syev_work_bytes(k, m) bytes.
size_t small_syev_work_bytes(int k, int m);
eig_status small_syev(const double* A, int k, int m, double* w, double* Z, void* work, int* info, cudaStream_t st);

// Lowest m eigenpairs of the symmetric tridiagonal (d[k], e[k-1]); Z (k x m row-major).
// work: small_syev_work_bytes(k, m).
eig_status small_tri_eig(const double* d, const double* e, int k, int m, double* w, double* Z, void* work,
                         cudaStream_t st);

// Rayleigh-Ritz on the pencil (A, G) = (S^T H S, S^T S) of Eq. (rreig), k x k, lowest nb:
// scales G to unit diagonal, Cholesky G = L L^T (breakdown when a squared pivot falls below
// piv_tol), T = L^{-1} A L^{-T}, T Z = Z Theta, C = D^{-1/2} L^{-T} Z.
// Outputs theta[nb], C (k x nb, row-major), C32 (optional float copy), info.
// pivoted = 1: a rank-revealing (diagonally pivoted) Cholesky of the scaled G first takes the
// basis columns in order of largest remaining pivot while it stays above piv_tol, and the
// Rayleigh-Ritz runs on those columns (the others get zero rows in C); breakdown only when
// fewer than nb columns remain.  For bases that lost rank (LOBPCG's [X W P] near convergence).
size_t small_rr_work_bytes(int k, int nb);
eig_status small_rr(const double* A, const double* G, int k, int nb, double piv_tol, double* theta, double* C,
                    float* C32, void* work, int* info, cudaStream_t st, int pivoted = 0);

// CholQR factor: G = R^T R (upper R) and Rinv = R^{-1}, k x k; info = SMALL_BREAKDOWN when a
// squared pivot falls below piv_tol * max diag(G).  Rinv32: optional float copy.
// work: small_chol_inv_work_bytes(k) bytes of device scratch.
size_t small_chol_inv_work_bytes(int k);
eig_status small_chol_inv(const double* G, int k, double piv_tol, double* R, double* Rinv, float* Rinv32,
                          void* work, int* info, cudaStream_t st);

}  // namespace eig
