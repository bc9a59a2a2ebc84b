// Learned per-row preconditioner (internal interface): w_ij = m_ij r_ij with m = J (1 + o),
// o = MLP(6 features) and J = 1 / floor(H_ii - theta_j) the Jacobi scale (|.| floored at
// kLpJacobiFloor, sign kept), so that a zero output layer is exactly the Jacobi K.
// Features of row i, column j: H_ii, theta_j, H_ii - theta_j, (|H| 1)_i, sqrt(n) r_ij / ||r_j||,
// sqrt(n) ((H - D) r_j)_i / ||r_j||.  Network 6 -> 32 -> 32 -> 1 (ReLU, FP32) on standardised
// features (f - mu) / sigma.  Flat FP32 parameters:
//   mu[6] sigma[6] | W1[32][6] b1[32] W2[32][32] b2[32] w3[32] b3
#pragma once
#include "common.cuh"
#include "spmm.cuh"

namespace eig {

constexpr int kLpFeat = 6, kLpHid = 32;
constexpr int kLpOffMu = 0, kLpOffSigma = 6, kLpFixed = 12;
constexpr int kLpOffW1 = 12;
constexpr int kLpOffB1 = kLpOffW1 + kLpHid * kLpFeat;   // 204
constexpr int kLpOffW2 = kLpOffB1 + kLpHid;             // 236
constexpr int kLpOffB2 = kLpOffW2 + kLpHid * kLpHid;    // 1260
constexpr int kLpOffW3 = kLpOffB2 + kLpHid;             // 1292
constexpr int kLpOffB3 = kLpOffW3 + kLpHid;             // 1324
constexpr int kLpParams = kLpOffB3 + 1;                 // 1325
constexpr int kLpTrained = kLpParams - kLpFixed;        // 1313
constexpr float kLpJacobiFloor = 2.0f;

// Passed by value: a kernel reads it from the constant bank of its parameters.
struct LpParams {
  float p[kLpParams];
};

// (|H| 1)_i of the full symmetric H from the plan's half-stored CSR: fixed-point (integer)
// accumulation, so the result does not depend on the order of the additions.
eig_status lp_row_abs_sum(const SpmmPlan& P, double* out, cudaStream_t st);

// W = m * R on the first m columns of n x ld blocks (vt F32 or F64), m from the features of
// (R, HR); entries whose product is not finite take the Jacobi value r / floor(d - theta).
// W may alias R.  rsq[j] = ||r_j||^2 (FP64, device), theta device FP64.  active (device int[m],
// may be null): a column with active[j] == 0 gets W = 0.  *nonfinite (device int, may be null)
// counts the Jacobi replacements.
eig_status lp_apply(const LpParams& prm, const void* R, const void* HR, int ld, int m, int64_t n, eig_dtype vt,
                    const double* diagH, const double* rowabs, const double* theta, const double* rsq, double floor_,
                    const int* active, void* W, int* nonfinite, cudaStream_t st);

// Feature rows F[(i*m + j)*6 + q] (FP32) and r (FP32, i*m + j) of the first m columns.
eig_status lp_features(const void* R, const void* HR, int ld, int m, int64_t n, eig_dtype vt, const double* diagH,
                       const double* rowabs, const double* theta, const double* rsq, float* F, float* r,
                       cudaStream_t st);

// m = J (1 + o) for count feature rows (FP32).
eig_status lp_forward(const LpParams& prm, const float* F, int64_t count, float* m_out, cudaStream_t st);

// Loss of the correction targets and its gradient (FP64 out[kLpTrained + 1]: the trained
// parameters' gradient, then the loss), for count = n*m entries with column weights colw[m].
size_t lp_grad_workspace_bytes();
eig_status lp_grad(const float* params, const float* F, const float* r, const float* z, const double* colw,
                   int64_t n, int m, double* out, void* workspace, cudaStream_t st);

// Adam step on the trained parameters (index >= 12) with grad from lp_grad.
eig_status lp_adam(float* params, const double* grad, float* m1, float* m2, int t, double lr, double beta1,
                   double beta2, double eps, cudaStream_t st);

}  // namespace eig
