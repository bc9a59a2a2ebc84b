// Tall-skinny dense kernels around the SpMM (internal interface).
#pragma once
#include "common.cuh"

namespace eig {

constexpr int kMaxBlocks = 64;   // blocks in one gram / apply call
constexpr int kMaxPairs = 16;    // block pairs in one gram call

struct BlockList {
  const void* p[kMaxBlocks];
  int n;
};

// G_q = A_{a_q}^T A_{b_q} for q < npairs, each nb x nb, FP64 out (G + q*nb*nb).  Blocks are
// n x nb row-major of vec type vt.  FP32 blocks: FP32 products summed in FP32 over 32-row
// chunks, chunk sums accumulated in double-float (hi+lo FP32 pairs), CTA partials in FP64.
// part: device scratch of gram_scratch_bytes(npairs, nb) bytes, or of max_parts * npairs * nb * nb
// doubles when max_parts > 0 caps the number of CTA partials.
size_t gram_scratch_bytes(int npairs, int nb);
eig_status gram_multi(const BlockList& blocks, const int* pa, const int* pb, int npairs, int nb, int64_t n,
                      eig_dtype vt, double* G, void* part, cudaStream_t st, int max_parts = 0);

// Out (n x m) = sum_s In_s (n x nb) * M[s*nb:(s+1)*nb, :]  (M FP64, K x m with K = nin*nb),
// optionally + beta * Out.  m <= 64, K <= 1024.
eig_status block_apply(const BlockList& in, int nb, const double* M, int m, void* Out, double beta, int64_t n,
                       eig_dtype vt, cudaStream_t st);

// Elementwise conversions / copies of n*k elements.
eig_status convert(const void* src, eig_dtype st_, void* dst, eig_dtype dt_, int64_t count, cudaStream_t st);

// Per-column sums of squares of an n x k block -> out[k] (FP64).
eig_status col_sumsq(const void* X, int k, int64_t n, eig_dtype vt, double* out, void* part, cudaStream_t st);
size_t colsum_scratch_bytes(int k);

// Fixed-order reduction of CTA partials: out[j] = sum_b part[b*m + j], b < nparts.
eig_status reduce_partials(const double* part, int nparts, int m, double* out, cudaStream_t st);

// LOBPCG fused update (Eqs. xupd, pupd, upd1, upd2, wblock):
//   P' = W C2 + P C3, HP' = HW C2 + HP C3, X' = X C1 + P', HX' = HX C1 + HP',
//   R = HX' - X' Theta, W' = K^{-1} R (Jacobi: r / (d_i - theta_j), |den| floored), and
//   per-column ||R_j||^2 partials.  C (k x nb FP64) has k = nb (no W, P), 2nb (no P) or 3nb.
//   X, P, HX, HP, W are updated in place.  With k == nb the call only forms R/W' from X, HX.
eig_status lobpcg_update(void* X, void* W, void* P, void* HX, void* HW, void* HP, const double* C, int k, int nb,
                         const double* theta, const double* diagH, double floor, int precond, int64_t n,
                         eig_dtype vt, double* part, int nparts_max, int* nparts_out, cudaStream_t st);
int update_grid(int64_t n);

// Jacobi preconditioner on a block: W = R / (d_i - theta_j) (floored), in place.
eig_status jacobi_block(void* R, const double* theta, const double* diagH, double floor, int nb, int64_t n,
                        eig_dtype vt, cudaStream_t st);

}  // namespace eig
