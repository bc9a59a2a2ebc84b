// Batched RMM-DIIS kernels (Alg. 4; Sec. 4.3 batches the n_ev refinements into one SpMM).
#pragma once
#include "common.cuh"

namespace eig {

constexpr int kRmmSMax = 20;  // largest DIIS window (the paper uses s_max = 10..20)

// Window of history slots, oldest first; slots index the ring buffers.
struct Window {
  int slot[kRmmSMax];
  int s;
};

// Combine (Eq. xsum) for every column j:  x~ = sum_i a_ji x^(i),
// Hx~ = sum_i a_ji (r^(i) + theta^(i) x^(i)),  r~ = Hx~ - theta_ref_j x~ (stored in the SpMM
// vector type; zero for inactive columns), and partial dots <x~,x~>, <x~,Hx~>, <x~,r~>, <r~,r~>,
// <r~,Hx~> (partials [cta][j][5]).
// xh: [s_max][n][mp] FP64; rh: [s_max][n][mp] (vt); thh: [s_max][mp]; alpha: [mp][kRmmSMax].
eig_status rmm_combine(const double* xh, const void* rh, const double* thh, const double* alpha, Window win,
                       const double* theta_ref, const int* active, int mp, int64_t n, eig_dtype vt, double* xt,
                       double* hxt, void* rt, double* part, int* nparts, cudaStream_t st);

// Preconditioned correction r~ = K^{-1}(H x~ - theta~ x~) with theta~ the Rayleigh quotient of x~
// (from the combine sums, stride 5) and the Jacobi K of the LOBPCG step; zero for inactive columns.
eig_status rmm_precond_resid(const double* xt, const double* hxt, const double* sums, const int* active,
                             const double* diagH, double floor, int mp, int64_t n, eig_dtype vt, void* rt,
                             cudaStream_t st);

// Partial dots <x~, H r~>, <r~, H r~>.
eig_status rmm_dots2(const double* xt, const void* rt, const void* hrt, int mp, int64_t n, eig_dtype vt, double* part,
                     int* nparts, cudaStream_t st);

// 2x2 Rayleigh-Ritz (Eqs. rr, xuwg) per column from the six dots (dots: [mp][6] = <x,x>, <x,Hx>,
// <x,r>, <r,r>, <x,Hr>, <r,Hr>): theta (lower root of the pencil) and g = (g1, g2) with
// g^T (W^T W) g = 1 and g1 <= 0.  Inactive columns get g = (1/||x~||, 0), theta = <x,Hx>/<x,x>.
eig_status rmm_rr2(const double* dots, const int* active, int mp, double* theta, double* g, cudaStream_t st);

// Update (Eq. xuwg): x = g1 x~ + g2 r~, Hx = g1 Hx~ + g2 H r~, r = Hx - theta x, written to the
// history slot `slot_new` (x FP64, r in vt); partials of ||r||^2 (FP64 r) and of
// <r, r^(i)> for the slots of `win_after` (the window including the new slot).
eig_status rmm_update(const double* xt, const double* hxt, const void* rt, const void* hrt, const double* g,
                      const double* theta, int slot_new, Window win_after, int mp, int64_t n, eig_dtype vt,
                      double* xh, void* rh, double* thh, double* part, int* nparts, cudaStream_t st);

// Start of Alg. 4 (lines 2-4) from a given (x, Hx): theta = num/xnorm2 with num = <x,Hx>,
// x/||x|| written to xh[slot], r = (Hx - theta x)/||x|| to rh[slot] (vt), theta to thh[slot]
// and theta_out; partials [cta][j][2] of ||r||^2 (FP64 r) and <rq, rq> (rounded r).
eig_status rmm_start(double* x, const double* hx, const double* num, const double* xnorm2, int mp, int64_t n,
                     eig_dtype vt, int slot, double* xh, void* rh, double* thh, double* theta_out, double* part,
                     int* nparts, cudaStream_t st);

// DIIS least squares (Eqs. alphasum, rmm) by the substitution alpha_last = 1 - sum(others):
// Cholesky of the (s-1)x(s-1) normal matrix of the residual differences, dropping the oldest
// entries while it is numerically singular.  B: [mp][kRmmSMax][kRmmSMax] Gram of the residual
// history by slot.  Inactive columns get alpha = one-hot on the newest slot.
// tol: an entry is dropped while a squared Cholesky pivot falls below tol * max diag (the normal
// matrix is only as accurate as the residual history it is built from).
eig_status rmm_diis(const double* B, Window win, const int* active, int mp, double* alpha, cudaStream_t st,
                    double tol = 1e-13);

// B[j][slot_new][slot_i] = B[j][slot_i][slot_new] = sums[j][1 + i] for i < win.s (sums: [mp][1+kRmmSMax]).
eig_status rmm_store_gram(double* B, const double* sums, Window win_after, int slot_new, int mp, cudaStream_t st);

int rmm_grid(int64_t n, int mp);

// ---- FP32-vector step (rmm_mixed.cu): iterates in double-float (float2 per element), residual
// history and every small quantity in FP32, dots in double-float then FP64; see that file. ----
int rmx_grid(int64_t n, int mp);
// Alg. 4 start from FP64 (x, Hx): x/||x|| as double-float into xh[slot], r (FP32) into rh[slot],
// theta; partials [cta][j][2] of ||r||^2 (twice: the first row of the Gram store).
eig_status rmx_start(const double* x0, const double* hx0, const double* num, const double* xnorm2, int mp, int64_t n,
                     int slot, void* xh, float* rh, double* thh, double* theta_out, double* part, int* nparts,
                     cudaStream_t st);
// x~ and r_raw = H x~ - theta_ref x~ from the window (coef: [mp][3 kRmmSMax] from rmx_coef);
// when w is given, w = r_raw for active columns and 0 otherwise; partials [cta][j][3] of
// <x~,x~>, <x~,r_raw>, <x~, y^(newest)>.
eig_status rmx_combine(const void* xh, const float* rh, const float* coef, Window win, int newest, const int* active,
                       int mp, int64_t n, void* xt, float* rraw, float* w, double* part, int* nparts,
                       cudaStream_t st);
// The combine coefficients from the DIIS alpha, the Ritz values and the storage signs sg
// ([kRmmSMax][mp], +-1) of the window.
eig_status rmx_coef(const double* alpha, const double* thh, const double* sg, Window win, int newest, int mp,
                    float* coef, cudaStream_t st);
// Residual Gram row of the new slot with the storage signs applied.
eig_status rmx_store_gram(double* B, const double* sums, const double* sg, Window win_after, int slot_new, int mp,
                          cudaStream_t st);
// w = K^{-1}(H x~ - theta~ x~) (Jacobi, floored) from the combine sums [mp][3].
// r~ = r_raw - mu x~ (FP32 n x mp, zero on inactive columns) and theta~ = theta_ref + mu (mp).
eig_status rmx_shifted(const void* xt, const float* rraw, const double* sums, const double* theta_ref,
                       const int* active, int mp, int64_t n, float* rt, double* theta_out, cudaStream_t st);
eig_status rmx_precond(const void* xt, const float* rraw, const double* sums, const double* theta_ref,
                       const int* active, const double* diagH, double floor_, int mp, int64_t n, float* w,
                       cudaStream_t st);
// partials [cta][j][5]: <x~,w>, <w,w>, <w,r_raw>, <x~,Hw - theta_ref w>, <w,Hw - theta_ref w>.
eig_status rmx_dots(const void* xt, const float* w, const float* rraw, const float* hw, const double* theta_ref,
                    int mp, int64_t n, double* part, int* nparts, cudaStream_t st);
// Shifted 2x2 Rayleigh-Ritz; theta and par[mp][5] = (g1, g2, mu, theta, storage sign).
eig_status rmx_rr2(const double* s1, const double* s2, const double* theta_ref, const int* active, int mp,
                   double* theta, double* par, cudaStream_t st);
// New iterate and residual (times the storage sign) into slot_new; partials [cta][j][1 + win.s] of
// ||r||^2 and <ry_new, ry^(i)>.
eig_status rmx_update(const void* xt, const float* w, const float* rraw, const float* hw, const double* par,
                      int slot_new, Window win_after, int mp, int64_t n, void* xh, float* rh, double* thh, double* sg,
                      double* part, int* nparts, cudaStream_t st);
// X (FP64, n x nev) = sign * (hi + lo) of the double-float iterate slot (n x mp).
eig_status rmx_export(const void* xh_slot, const double* sgn, int mp, int nev, int64_t n, double* X, cudaStream_t st);

}  // namespace eig
