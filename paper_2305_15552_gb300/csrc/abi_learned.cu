// C ABI of the learned per-row preconditioner: training samples from the solver's matrix,
// inference, loss gradient and Adam step (the network and features are in learned.cuh).
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dense.cuh"
#include "learned.cuh"
#include "solver.cuh"

namespace eig {

eig_status lp_ensure_rowabs(Handle* h, cudaStream_t st) {
  if (h->lp_rowabs_ok) return EIG_OK;
  EIG_TRY(h->lp_rowabs.reserve((size_t)h->n * 8));
  EIG_TRY(lp_row_abs_sum(h->plan, h->lp_rowabs.as<double>(), st));
  h->lp_rowabs_ok = true;
  return EIG_OK;
}

namespace {

// R = HX - X diag(theta) over n x ld (FP64)
__global__ void k_lp_resid(const double* __restrict__ X, const double* __restrict__ HX,
                           const double* __restrict__ th, int ld, int64_t n, double* __restrict__ R) {
  const int64_t cnt = n * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    R[e] = HX[e] - X[e] * th[e % ld];
}

// CTA partials of P = Xs^T X (k x m): part[cta][a*m + b]
__global__ void k_lp_cross(const double* __restrict__ Xs, int k, const double* __restrict__ X, int m, int64_t n,
                           double* __restrict__ part) {
  const int per = k * m;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = blockIdx.x * chunk, r1 = min64(n, r0 + chunk);
  for (int o = threadIdx.x; o < per; o += blockDim.x) {
    const int a = o / m, b = o % m;
    double s = 0.0;
    for (int64_t i = r0; i < r1; ++i) s += Xs[i * k + a] * X[i * m + b];
    part[(size_t)blockIdx.x * per + o] = s;
  }
}

// z (n x m): target 0: x_j - Xs P_j / |P_j|^2; target 1: r / floor(d - theta).  z64 and z32.
__global__ void k_lp_target(int target, const double* __restrict__ X, int m, const double* __restrict__ Xs, int k,
                            const double* __restrict__ P, const double* __restrict__ R, int ldr,
                            const double* __restrict__ diagH, const double* __restrict__ th, double floor_, int64_t n,
                            double* __restrict__ z64, float* __restrict__ z32) {
  __shared__ double sC[32 * 32];
  __shared__ double sTh[32];
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    sTh[j] = th[j];
    if (target == 0) {
      double s = 0.0;
      for (int a = 0; a < k; ++a) s += P[a * m + j] * P[a * m + j];
      for (int a = 0; a < k; ++a) sC[a * m + j] = s > 0.0 ? P[a * m + j] / s : 0.0;
    }
  }
  __syncthreads();
  const int64_t cnt = n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m;
    const int j = (int)(e - i * m);
    double z;
    if (target == 0) {
      z = X[e];
      for (int a = 0; a < k; ++a) z -= Xs[i * k + a] * sC[a * m + j];
      bool any = false;
      for (int a = 0; a < k; ++a) any = any || sC[a * m + j] != 0.0;
      if (!any) z = 0.0;
    } else {
      double den = diagH[i] - sTh[j];
      const double mag = fmax(fabs(den), floor_);
      den = den < 0.0 ? -mag : mag;
      z = R[i * ldr + j] / den;
    }
    z64[e] = z;
    z32[e] = (float)z;
  }
}

// colw_j = 1 / (|J| ||z_j||^2) over the columns with a target
__global__ void k_lp_colw(const double* __restrict__ zz, const double* __restrict__ P, int k, int m, int target,
                          double* __restrict__ colw) {
  if (threadIdx.x != 0) return;
  int nJ = 0;
  bool ok[32];
  for (int j = 0; j < m; ++j) {
    double s = 1.0;
    if (target == 0) {
      s = 0.0;
      for (int a = 0; a < k; ++a) s += P[a * m + j] * P[a * m + j];
    }
    ok[j] = s > 0.0 && zz[j] > 0.0;
    nJ += ok[j];
  }
  for (int j = 0; j < m; ++j) colw[j] = ok[j] ? 1.0 / ((double)nJ * zz[j]) : 0.0;
}

void load_params(const float* host, LpParams* p) { std::memcpy(p->p, host, sizeof(p->p)); }

}  // namespace
}  // namespace eig

using namespace eig;

extern "C" {

int eig_lp_param_count(void) { return kLpParams; }

eig_status eig_lp_sample(void* handle, const double* X, int m, const double* theta, const double* Xstar, int k,
                         int target, double floor_, float* F, float* r, float* z, double* colw, void* stream) {
  Handle* h = static_cast<Handle*>(handle);
  if (!h || !X || !theta || !F || !r || !z || !colw) return EIG_EINVAL;
  if (m < 1 || m > 32 || (target != 0 && target != 1) || !(floor_ >= 0.0)) return EIG_EINVAL;
  if (target == 0 && (!Xstar || k < 1 || k > 32)) return EIG_EINVAL;
  if (target == 1) k = 0;
  cudaStream_t st = as_stream(stream);
  const int64_t n = h->n;
  const int mp = next_pow2(m);
  EIG_TRY(lp_ensure_rowabs(h, st));
  for (int b = 0; b < 3; ++b) EIG_TRY(h->lp_buf[b].reserve((size_t)n * mp * 8));
  const int grid = num_sms() * 2;
  const size_t part_bytes = std::max(colsum_scratch_bytes(mp), (size_t)grid * std::max(1, k * m) * 8);
  EIG_TRY(h->lp_small.reserve(4 * 32 * 8 + 32 * 32 * 8 + part_bytes + 4 * 256));
  unsigned char* sb = h->lp_small.as<unsigned char>();
  double* th_d = (double*)sb;
  double* rsq = th_d + 32;
  double* zz = rsq + 32;
  double* Pm = zz + 32;                              // k x m
  void* part = (void*)(((uintptr_t)(Pm + 32 * 32) + 255) & ~(uintptr_t)255);
  double *Xp = h->lp_buf[0].as<double>(), *HX = h->lp_buf[1].as<double>(), *R = h->lp_buf[2].as<double>();
  std::vector<double> thp(mp, 0.0);
  for (int j = 0; j < m; ++j) thp[j] = theta[j];
  EIG_CUDA_TRY(cudaMemcpyAsync(th_d, thp.data(), mp * 8, cudaMemcpyHostToDevice, st));
  EIG_TRY(pad_columns(X, m, Xp, mp, n, st));
  EIG_TRY(spmm_run(&h->plan, Xp, HX, mp, EIG_F64, st));
  const int eg = num_sms() * 8;
  k_lp_resid<<<eg, 256, 0, st>>>(Xp, HX, th_d, mp, n, R);
  EIG_LAUNCH_CHECK("k_lp_resid");
  EIG_TRY(col_sumsq(R, mp, n, EIG_F64, rsq, part, st));
  EIG_TRY(spmm_run(&h->plan, R, HX, mp, EIG_F64, st));   // H R
  EIG_TRY(lp_features(R, HX, mp, m, n, EIG_F64, h->plan.diag.as<double>(), h->lp_rowabs.as<double>(), th_d, rsq, F,
                      r, st));
  if (target == 0) {
    k_lp_cross<<<grid, 256, 0, st>>>(Xstar, k, X, m, n, (double*)part);
    EIG_LAUNCH_CHECK("k_lp_cross");
    EIG_TRY(reduce_partials((const double*)part, grid, k * m, Pm, st));
  }
  double* z64 = Xp;   // n x m, the padded X is no longer needed
  k_lp_target<<<eg, 256, 0, st>>>(target, X, m, Xstar, k, Pm, R, mp, h->plan.diag.as<double>(), th_d, floor_, n, z64,
                                  z);
  EIG_LAUNCH_CHECK("k_lp_target");
  EIG_TRY(col_sumsq(z64, m, n, EIG_F64, zz, part, st));
  k_lp_colw<<<1, 32, 0, st>>>(zz, Pm, k, m, target, colw);
  EIG_LAUNCH_CHECK("k_lp_colw");
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  return EIG_OK;
}

eig_status eig_lp_apply(void* handle, const float* params, const void* R, int m, eig_dtype vec_type,
                        const double* theta, double floor_, void* W, void* stream) {
  Handle* h = static_cast<Handle*>(handle);
  if (!h || !params || !R || !theta || !W) return EIG_EINVAL;
  if (m < 1 || m > 32 || (m & (m - 1)) || (vec_type != EIG_F32 && vec_type != EIG_F64)) return EIG_EINVAL;
  cudaStream_t st = as_stream(stream);
  const int64_t n = h->n;
  EIG_TRY(lp_ensure_rowabs(h, st));
  EIG_TRY(h->lp_buf[0].reserve((size_t)n * m * dtype_size(vec_type)));
  EIG_TRY(h->lp_small.reserve(2 * 32 * 8 + colsum_scratch_bytes(m) + 2 * 256));
  double* th_d = h->lp_small.as<double>();
  double* rsq = th_d + 32;
  void* part = (void*)(((uintptr_t)(rsq + 32) + 255) & ~(uintptr_t)255);
  EIG_CUDA_TRY(cudaMemcpyAsync(th_d, theta, m * 8, cudaMemcpyHostToDevice, st));
  EIG_TRY(col_sumsq(R, m, n, vec_type, rsq, part, st));
  EIG_TRY(spmm_run(&h->plan, R, h->lp_buf[0].p, m, vec_type, st));
  LpParams prm;
  load_params(params, &prm);
  EIG_TRY(lp_apply(prm, R, h->lp_buf[0].p, m, m, n, vec_type, h->plan.diag.as<double>(), h->lp_rowabs.as<double>(),
                   th_d, rsq, floor_, nullptr, W, nullptr, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  return EIG_OK;
}

eig_status eig_lp_forward(const float* params, const float* F, int64_t count, float* m_out, void* stream) {
  if (!params || (count > 0 && (!F || !m_out))) return EIG_EINVAL;
  LpParams prm;
  load_params(params, &prm);
  return lp_forward(prm, F, count, m_out, as_stream(stream));
}

size_t eig_lp_grad_workspace_bytes(void) { return lp_grad_workspace_bytes(); }

eig_status eig_lp_grad(const float* params, const float* F, const float* r, const float* z, const double* colw,
                       int64_t n, int m, double* grad, void* workspace, void* stream) {
  if (!params || !grad || !workspace || m < 1 || m > 32 || n < 0) return EIG_EINVAL;
  if (n > 0 && (!F || !r || !z || !colw)) return EIG_EINVAL;
  return lp_grad(params, F, r, z, colw, n, m, grad, workspace, as_stream(stream));
}

eig_status eig_lp_adam(float* params, const double* grad, float* m1, float* m2, int t, double lr, double beta1,
                       double beta2, double eps, void* stream) {
  if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return EIG_EINVAL;
  return lp_adam(params, grad, m1, m2, t, lr, beta1, beta2, eps, as_stream(stream));
}

}  // extern "C"
