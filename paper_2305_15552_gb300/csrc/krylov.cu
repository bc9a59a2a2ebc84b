// Lanczos with full orthogonalisation (Sec. 2.1), block Lanczos (Alg. 1) and Chebyshev-filtered
// subspace iteration (Alg. 3), plus the lambda_ub estimate of Sec. 3.2.
//
// Lanczos keeps its basis column-major (each v_j contiguous): the SpMV is the SpMM with nb = 1,
// and the projections V^T w and w - V c are single passes over the basis (multi-dot and
// multi-axpy kernels).  Block Lanczos keeps n x nb row-major blocks and reuses the Gram /
// block-apply kernels.  The Chebyshev three-term recurrence is a fused elementwise pass.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "dense.cuh"
#include "small.cuh"
#include "solver.cuh"
#include "spmm.cuh"

namespace eig {

eig_status cholqr2_impl2(void* X, void* X2, int64_t n, int k, eig_dtype vt, double* R, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------------------
constexpr int kMdRows = 2048;

// part[cta][c] = sum over the CTA's rows of V[c][r] * w[r]  (V column-major, ld = n)
template <typename T>
__global__ void k_multidot(const T* __restrict__ V, int j, const T* __restrict__ w, int64_t n, int64_t rpc,
                           double* __restrict__ part) {
  __shared__ double sw[kMdRows];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t r0 = blockIdx.x * rpc, r1 = min64(n, r0 + rpc);
  double* out = part + (size_t)blockIdx.x * j;
  for (int c = threadIdx.x; c < j; c += blockDim.x) out[c] = 0.0;
  __syncthreads();
  for (int64_t rc = r0; rc < r1; rc += kMdRows) {
    const int rows = (int)min64(kMdRows, r1 - rc);
    __syncthreads();
    for (int i = threadIdx.x; i < rows; i += blockDim.x) sw[i] = (double)w[rc + i];
    __syncthreads();
    for (int c = wp; c < j; c += nw) {
      const T* v = V + (size_t)c * n + rc;
      double acc = 0.0;
      for (int i = lane; i < rows; i += 32) acc = fma((double)v[i], sw[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) out[c] += acc;
    }
  }
}

// w[r] -= sum_c V[c][r] * coef[c]
template <typename T>
__global__ void k_multiaxpy(T* __restrict__ w, const T* __restrict__ V, int j, const double* __restrict__ coef,
                           int64_t n) {
  extern __shared__ double sc[];
  for (int c = threadIdx.x; c < j; c += blockDim.x) sc[c] = coef[c];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double acc = (double)w[r];
    for (int c = 0; c < j; ++c) acc = fma(-(double)V[(size_t)c * n + r], sc[c], acc);
    w[r] = (T)acc;
  }
}

// out (n x m, FP64 row-major) = V[:, :k] Z, Z (k x m row-major)
template <typename T>
__global__ void k_basis_combine(const T* __restrict__ V, int k, const double* __restrict__ Z, int m, int64_t n,
                                double* __restrict__ out) {
  extern __shared__ double sz[];
  for (int i = threadIdx.x; i < k * m; i += blockDim.x) sz[i] = Z[i];
  __syncthreads();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double acc[32];
    for (int t = 0; t < m; ++t) acc[t] = 0.0;
    for (int c = 0; c < k; ++c) {
      const double v = (double)V[(size_t)c * n + r];
      for (int t = 0; t < m; ++t) acc[t] = fma(v, sz[c * m + t], acc[t]);
    }
    for (int t = 0; t < m; ++t) out[r * m + t] = acc[t];
  }
}

// d[j] = alpha (sum of two CGS passes' own coefficient), e[j] = beta
__global__ void k_lanczos_coef(const double* __restrict__ c1, const double* __restrict__ c2, const double* __restrict__ bb,
                               int j, double* __restrict__ d, double* __restrict__ e) {
  if (threadIdx.x == 0) {
    d[j] = c1[j] + c2[j];
    e[j] = sqrt(fmax(bb[0], 0.0));
  }
}

template <typename T>
__global__ void k_scale_into(const T* __restrict__ src, T* __restrict__ dst, const double* __restrict__ nrm2,
                             int64_t n) {
  const double s = rsqrt(fmax(nrm2[0], 1e-300));
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    dst[r] = (T)((double)src[r] * s);
}

// Columns of X (and X2) scaled by 1 / sqrt(nrm2[j])
template <typename T>
__global__ void k_scale_cols(T* __restrict__ X, T* __restrict__ X2, const double* __restrict__ nrm2, int k,
                             int64_t n) {
  const int64_t total = n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % k);
    const double s = rsqrt(fmax(nrm2[j], 1e-300));
    X[i] = (T)((double)X[i] * s);
    if (X2) X2[i] = (T)((double)X2[i] * s);
  }
}

// Chebyshev recurrence on active columns (Eq. chebypoly, Alg. 3 lines 5 and 7):
//   first:  Y = (HW - c W) / e
//   later:  Y = 2 (HW - c W) / e - Qp
// inactive (locked) columns: Y = W.
template <typename T>
__global__ void k_cheb(const T* __restrict__ HW, const T* __restrict__ W, const T* __restrict__ Qp, T* __restrict__ Y,
                       const int* __restrict__ active, double c, double e, int first, int k, int64_t n) {
  const int64_t total = n * k;
  const double a = first ? 1.0 / e : 2.0 / e;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % k);
    if (!active[j]) { Y[i] = W[i]; continue; }
    // explicit roundings (no contraction left to the compiler): the fused SpMM epilogue
    // evaluates the same expression the same way, so both give the same bits
    double y = __dmul_rn(a, __fma_rn(-c, (double)W[i], (double)HW[i]));
    if (!first) y = __dsub_rn(y, (double)Qp[i]);
    Y[i] = (T)y;
  }
}

// Per-column partials of ||HQ_j - theta_j Q_j||^2
template <typename T>
__global__ void k_resid_sumsq(const T* __restrict__ Q, const T* __restrict__ HQ, const double* __restrict__ theta,
                              int k, int64_t n, double* __restrict__ part) {
  __shared__ double red[256];
  const int j = threadIdx.x % k, rr = threadIdx.x / k, rpp = blockDim.x / k;
  double s = 0.0;
  if (rr < rpp) {
    const double th = theta[j];
    for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
      const double v = (double)HQ[r * k + j] - th * (double)Q[r * k + j];
      s = fma(v, v, s);
    }
  }
  red[threadIdx.x] = (rr < rpp) ? s : 0.0;
  __syncthreads();
  if (threadIdx.x < k) {
    double t = 0.0;
    for (int q = 0; q < rpp; ++q) t += red[q * k + threadIdx.x];
    part[(size_t)blockIdx.x * k + threadIdx.x] = t;
  }
}

// Exact block-Lanczos residual estimate ||R_{i+1} E_i^T q_t|| / |theta_t| (Eq. ritzest2, exact form):
// R (nb x nb), Zl = last nb rows of Z (nb x m row-major within Z of width m).
__global__ void k_block_est(const double* __restrict__ R, const double* __restrict__ Z, int k, int nb, int m,
                            const double* __restrict__ theta, double* __restrict__ est, double* __restrict__ est_paper,
                            double wnorm_f) {
  const int t = threadIdx.x;
  if (t >= m) return;
  double s = 0.0, ez = 0.0;
  for (int i = 0; i < nb; ++i) {
    double v = 0.0;
    for (int l = 0; l < nb; ++l) v += R[i * nb + l] * Z[(size_t)(k - nb + l) * m + t];
    s += v * v;
    const double z = Z[(size_t)(k - nb + i) * m + t];
    ez += z * z;
  }
  const double at = fmax(fabs(theta[t]), 1e-300);
  est[t] = sqrt(s) / at;
  est_paper[t] = wnorm_f * sqrt(ez) / at;
}

// T (ld x ld) diagonal block i <- sym(A), sub/super block (i+1, i) <- R / R^T
__global__ void k_put_blocks(double* __restrict__ T, int ld, int i, int nb, const double* __restrict__ A,
                             const double* __restrict__ R) {
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int a = e / nb, b = e % nb;
    if (A) T[(size_t)(i * nb + a) * ld + i * nb + b] = 0.5 * (A[a * nb + b] + A[b * nb + a]);
    if (R) {
      T[(size_t)((i + 1) * nb + a) * ld + i * nb + b] = R[a * nb + b];
      T[(size_t)(i * nb + b) * ld + (i + 1) * nb + a] = R[a * nb + b];
    }
  }
}

// After a thick restart: the couplings of the kept Ritz vectors (blocks 0..q-1) to block q,
// C_b = V_b^T H V_q, into T's column block q and row block q.
__global__ void k_put_coupling(double* __restrict__ T, int ld, int q, int nb, const double* __restrict__ C) {
  const int tot = q * nb * nb;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < tot; e += blockDim.x * gridDim.x) {
    const int b = e / (nb * nb), a = (e / nb) % nb, col = e % nb;
    const double v = C[e];
    T[(size_t)(b * nb + a) * ld + q * nb + col] = v;
    T[(size_t)(q * nb + col) * ld + b * nb + a] = v;
  }
}

// T (ld x ld, zeroed by the caller) <- diag(theta_0 .. theta_{p-1}) in its leading p x p
__global__ void k_set_diag(double* __restrict__ T, int ld, const double* __restrict__ theta, int p) {
  for (int i = threadIdx.x; i < p; i += blockDim.x) T[(size_t)i * ld + i] = theta[i];
}

// copy the leading k x k of a matrix with leading dimension ld into a dense k x k
__global__ void k_copy_lead(const double* __restrict__ T, int ld, int k, double* __restrict__ out) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < k * k; e += blockDim.x * gridDim.x)
    out[e] = T[(size_t)(e / k) * ld + e % k];
}

static int md_grid(int64_t n, int64_t* rpc) {
  int g = num_sms() * 2;
  int64_t r = (n + g - 1) / g;
  if (r < 256) r = 256;
  g = (int)((n + r - 1) / r);
  *rpc = r;
  return g;
}

// ---------------------------------------------------------------------------------------
// Lanczos machinery (shared by run_lanczos and the lambda_ub estimate)
// ---------------------------------------------------------------------------------------
struct LanczosState {
  int64_t n;
  eig_dtype vt;
  size_t sv;
  void* V;          // column-major basis, maxb + 1 columns
  void* w;          // n
  int maxb;
  double *d, *e, *c1, *c2, *bb, *part, *wr, *Z, *work;
};

static eig_status lanczos_alloc(Ctx& c, int maxb, int m, LanczosState* L) {
  Handle* h = c.h;
  L->n = h->n;
  L->vt = c.o.vec_type;
  L->sv = dtype_size(L->vt);
  L->maxb = maxb;
  int64_t rpc;
  const int g = md_grid(L->n, &rpc);
  const size_t big = (size_t)(maxb + 2) * L->n * L->sv + 512;
  EIG_TRY(h->big.reserve(big));
  L->V = h->big.p;
  L->w = (unsigned char*)h->big.p + (size_t)(maxb + 1) * L->n * L->sv;
  const size_t sm = (size_t)maxb * 8 * 4 + (size_t)g * (maxb + 1) * 8 + (size_t)maxb * m * 8 +
                    small_syev_work_bytes(maxb, m) + 64 * 256;
  EIG_TRY(h->small.reserve(sm));
  unsigned char* p = (unsigned char*)h->small.p;
  auto take = [&](size_t b) { unsigned char* r = p; p += (b + 255) & ~size_t(255); return r; };
  L->d = (double*)take(maxb * 8);
  L->e = (double*)take(maxb * 8);
  L->c1 = (double*)take((maxb + 1) * 8);
  L->c2 = (double*)take((maxb + 1) * 8);
  L->bb = (double*)take(64);
  L->wr = (double*)take(256 * 8);
  L->Z = (double*)take((size_t)maxb * m * 8);
  L->part = (double*)take((size_t)g * (maxb + 1) * 8);
  L->work = (double*)take(small_syev_work_bytes(maxb, m));
  return EIG_OK;
}

template <typename T>
static eig_status proj_pass(LanczosState& L, int j, double* coef, cudaStream_t st) {
  int64_t rpc;
  const int g = md_grid(L.n, &rpc);
  k_multidot<T><<<g, 256, 0, st>>>((const T*)L.V, j, (const T*)L.w, L.n, rpc, L.part);
  EIG_LAUNCH_CHECK("k_multidot");
  EIG_TRY(reduce_partials(L.part, g, j, coef, st));
  k_multiaxpy<T><<<num_sms() * 8, 256, (size_t)j * 8, st>>>((T*)L.w, (const T*)L.V, j, coef, L.n);
  EIG_LAUNCH_CHECK("k_multiaxpy");
  return EIG_OK;
}

// One Lanczos step j (0-based): w = H v_j, CGS2 against v_0..v_j, alpha_j, beta_j; writes d[j], e[j].
static eig_status lanczos_step(Ctx& c, LanczosState& L, int j) {
  void* vj = (unsigned char*)L.V + (size_t)j * L.n * L.sv;
  EIG_TRY(c.spmm(vj, L.w, 1, L.vt, 1));
  if (L.vt == EIG_F32) {
    EIG_TRY(proj_pass<float>(L, j + 1, L.c1, c.st));
    EIG_TRY(proj_pass<float>(L, j + 1, L.c2, c.st));
  } else {
    EIG_TRY(proj_pass<double>(L, j + 1, L.c1, c.st));
    EIG_TRY(proj_pass<double>(L, j + 1, L.c2, c.st));
  }
  EIG_TRY(col_sumsq(L.w, 1, L.n, L.vt, L.bb, L.part, c.st));
  k_lanczos_coef<<<1, 32, 0, c.st>>>(L.c1, L.c2, L.bb, j, L.d, L.e);
  EIG_LAUNCH_CHECK("k_lanczos_coef");
  // v_{j+1} = w / beta_j
  void* vn = (unsigned char*)L.V + (size_t)(j + 1) * L.n * L.sv;
  if (L.vt == EIG_F32) k_scale_into<float><<<num_sms() * 8, 256, 0, c.st>>>((const float*)L.w, (float*)vn, L.bb, L.n);
  else k_scale_into<double><<<num_sms() * 8, 256, 0, c.st>>>((const double*)L.w, (double*)vn, L.bb, L.n);
  EIG_LAUNCH_CHECK("k_scale_into");
  return EIG_OK;
}

// v_0 = normalised mean of the first `cols` columns of X0 (Sec. 3.2), written to V[:, 0].
static eig_status lanczos_start(Ctx& c, LanczosState& L, const double* X0, int x0c, int cols) {
  DevBuf v64, M;
  EIG_TRY(v64.reserve((size_t)L.n * 8));
  EIG_TRY(M.reserve((size_t)x0c * 8));
  std::vector<double> hm(x0c, 0.0);
  for (int i = 0; i < std::min(cols, x0c); ++i) hm[i] = 1.0 / std::min(cols, x0c);
  EIG_CUDA_TRY(cudaMemcpyAsync(M.p, hm.data(), x0c * 8, cudaMemcpyHostToDevice, c.st));
  BlockList in;
  in.n = 1;
  in.p[0] = X0;
  EIG_TRY(block_apply(in, x0c, M.as<double>(), 1, v64.p, 0.0, L.n, EIG_F64, c.st));
  EIG_TRY(col_sumsq(v64.p, 1, L.n, EIG_F64, L.bb, L.part, c.st));
  DevBuf tmp;
  EIG_TRY(tmp.reserve((size_t)L.n * L.sv));
  EIG_TRY(convert(v64.p, EIG_F64, tmp.p, L.vt, L.n, c.st));
  if (L.vt == EIG_F32) k_scale_into<float><<<num_sms() * 8, 256, 0, c.st>>>((const float*)tmp.p, (float*)L.V, L.bb, L.n);
  else k_scale_into<double><<<num_sms() * 8, 256, 0, c.st>>>((const double*)tmp.p, (double*)L.V, L.bb, L.n);
  EIG_LAUNCH_CHECK("k_scale_into");
  EIG_TRY(c.sync());
  return EIG_OK;
}

eig_status run_lanczos(Ctx& c, const double* X0, int x0c, int* iters, bool* converged,
                       std::vector<double>* theta_out) {
  Handle* h = c.h;
  const int nev = h->n_ev;
  const int maxb = (int)std::min<int64_t>(std::max(c.o.lanczos_maxbasis, nev + 1), h->n);
  LanczosState L;
  EIG_TRY(lanczos_alloc(c, maxb, nev, &L));
  EIG_TRY(lanczos_start(c, L, X0, x0c, nev));
  EIG_TRY(h->host.reserve((size_t)(2 * nev + 8) * 8 + (size_t)nev * 8));
  double* hs = h->host.as<double>();
  *converged = false;
  int k = 0;
  std::vector<double> th(nev, 0.0);
  for (int j = 0; j < maxb; ++j) {
    EIG_TRY(lanczos_step(c, L, j));
    k = j + 1;
    const int m = std::min(nev, k);
    EIG_TRY(small_tri_eig(L.d, L.e, k, m, L.wr, L.Z, L.work, c.st));
    // Ritz values, last row of Z, beta_j
    EIG_CUDA_TRY(cudaMemcpyAsync(hs, L.wr, m * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs + nev, L.Z + (size_t)(k - 1) * m, m * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs + 2 * nev, L.e + j, 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    const double beta = hs[2 * nev];
    bool conv = (m == nev);
    double tn = 0.0;
    for (int t = 0; t < m; ++t) {
      th[t] = hs[t];
      tn = std::max(tn, std::fabs(hs[t]));
      const double est = beta * std::fabs(hs[nev + t]) / std::max(std::fabs(hs[t]), 1e-300);
      conv = conv && est < c.o.tol;
    }
    {
      std::vector<double> rr(m);
      for (int t = 0; t < m; ++t) rr[t] = beta * std::fabs(hs[nev + t]) / std::max(std::fabs(hs[t]), 1e-300);
      c.trace(0, k, th.data(), rr.data(), m);
    }
    if (conv) { *converged = true; break; }
    if (beta <= 1e-14 * std::max(1.0, tn)) { *converged = (m == nev); break; }  // invariant subspace
  }
  *iters = k;
  // X = V_k Z
  const int m = std::min(nev, k);
  EIG_TRY(h->Xres.reserve((size_t)h->n * nev * 8));
  EIG_CUDA_TRY(cudaMemsetAsync(h->Xres.p, 0, (size_t)h->n * nev * 8, c.st));
  if (m == nev) {
    const size_t sm = (size_t)k * m * 8;
    if (L.vt == EIG_F32) {
      EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_basis_combine<float>, 160 * 1024));
      k_basis_combine<float><<<num_sms() * 4, 256, sm, c.st>>>((const float*)L.V, k, L.Z, m, h->n, h->Xres.as<double>());
    } else {
      EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_basis_combine<double>, 160 * 1024));
      k_basis_combine<double><<<num_sms() * 4, 256, sm, c.st>>>((const double*)L.V, k, L.Z, m, h->n, h->Xres.as<double>());
    }
    EIG_LAUNCH_CHECK("k_basis_combine");
  }
  EIG_TRY(c.sync());
  theta_out->assign(th.begin(), th.end());
  return EIG_OK;
}

// lambda_ub = theta_max + ||r|| after `steps` Lanczos steps from a seeded random vector (Sec. 3.2)
static eig_status lambda_ub_estimate(Ctx& c, int steps, double* lub) {
  Handle* h = c.h;
  steps = (int)std::min<int64_t>(steps, h->n);
  LanczosState L;
  EIG_TRY(lanczos_alloc(c, steps, steps, &L));
  DevBuf r;
  EIG_TRY(r.reserve((size_t)h->n * 8));
  EIG_TRY(fill_random(r.as<double>(), h->n, c.o.seed + 101, c.st));
  EIG_TRY(lanczos_start(c, L, r.as<double>(), 1, 1));
  int k = 0;
  for (int j = 0; j < steps; ++j) {
    EIG_TRY(lanczos_step(c, L, j));
    k = j + 1;
  }
  EIG_TRY(small_tri_eig(L.d, L.e, k, k, L.wr, L.Z, L.work, c.st));
  std::vector<double> w(k), zl(k);
  double beta = 0.0;
  EIG_CUDA_TRY(cudaMemcpyAsync(w.data(), L.wr, k * 8, cudaMemcpyDeviceToHost, c.st));
  EIG_CUDA_TRY(cudaMemcpyAsync(zl.data(), L.Z + (size_t)(k - 1) * k, k * 8, cudaMemcpyDeviceToHost, c.st));
  EIG_CUDA_TRY(cudaMemcpyAsync(&beta, L.e + (k - 1), 8, cudaMemcpyDeviceToHost, c.st));
  EIG_TRY(c.sync());
  *lub = w[k - 1] + beta * std::fabs(zl[k - 1]);
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// block Lanczos (Alg. 1)
// ---------------------------------------------------------------------------------------
// C (count x nb x nb) = V_b^T Y for blocks b < count (chunks of 15 blocks per Gram call)
static eig_status basis_gram(Ctx& c, void* const* blocks, int count, const void* Y, int nb, eig_dtype vt, double* C,
                             void* gpart) {
  for (int b0 = 0; b0 < count; b0 += 15) {
    const int cnt = std::min(15, count - b0);
    BlockList bl;
    bl.n = cnt + 1;
    int pa[16], pb[16];
    for (int i = 0; i < cnt; ++i) { bl.p[i] = blocks[b0 + i]; pa[i] = i; pb[i] = cnt; }
    bl.p[cnt] = Y;
    EIG_TRY(gram_multi(bl, pa, pb, cnt, nb, c.h->n, vt, C + (size_t)b0 * nb * nb, gpart, c.st));
  }
  return EIG_OK;
}

__global__ void k_negate_stack(const double* __restrict__ C, int count, int nb, double* __restrict__ M) {
  // M = [-C_0; ...; -C_{count-1}; I]  ((count+1) nb x nb)
  const int tot = (count + 1) * nb * nb;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < tot; e += blockDim.x * gridDim.x) {
    const int row = e / nb, col = e % nb;
    M[e] = (row < count * nb) ? -C[e] : (row - count * nb == col ? 1.0 : 0.0);
  }
}

eig_status run_block_lanczos(Ctx& c, const double* X0, int x0c, int maxiter, const StopFn& stop, int* iters,
                             int* reason, bool* converged, std::vector<double>* theta_out) {
  Handle* h = c.h;
  const int nb = h->nb, nev = h->n_ev;
  const int64_t n = h->n;
  const eig_dtype vt = c.o.vec_type;
  const size_t sv = dtype_size(vt);
  const int maxblocks = std::max(2, std::min({c.o.lanczos_maxbasis / nb, 62, (int)(n / nb)}));
  // thick restart (Sec. 2.2): when the basis holds maxblocks blocks, keep the lowest `keep` Ritz
  // vectors (a multiple of nb, at least n_ev, leaving room for one more block) and continue
  const int nevb = ((nev + nb - 1) / nb) * nb;
  int keep = 0;
  if (c.o.lanczos_keep >= 0) {
    int kk = c.o.lanczos_keep > 0 ? ((c.o.lanczos_keep + nb - 1) / nb) * nb : (maxblocks / 2) * nb;
    kk = std::min(std::max(kk, nevb), 256 / nb * nb);
    if (kk >= nevb && kk <= (maxblocks - 1) * nb) keep = kk;
  }
  const int qkeep = keep / nb;
  const int mz = std::max(nev, keep);   // columns of Z: the wanted pairs, or the kept ones at a restart
  const size_t blk = (size_t)n * nb * sv;
  EIG_TRY(h->big.reserve((size_t)(maxblocks + 3 + qkeep) * blk + 512));
  std::vector<void*> V(maxblocks + 1);
  for (int b = 0; b <= maxblocks; ++b) V[b] = (unsigned char*)h->big.p + (size_t)b * blk;
  void* HV = (unsigned char*)h->big.p + (size_t)(maxblocks + 1) * blk;
  void* W = (unsigned char*)h->big.p + (size_t)(maxblocks + 2) * blk;
  unsigned char* Ytmp = (unsigned char*)h->big.p + (size_t)(maxblocks + 3) * blk;   // qkeep blocks
  const int kmax = maxblocks * nb;
  const size_t gsz = gram_scratch_bytes(15, nb);
  const size_t sm = (size_t)kmax * kmax * 8 * 2 + (size_t)(maxblocks + 1) * nb * nb * 8 * 2 + (size_t)kmax * mz * 8 +
                    small_syev_work_bytes(kmax, mz) + gsz + 256 * 8 * 3 + (size_t)nb * nb * 8 * 2 +
                    (size_t)kmax * nb * 8 + 5 * 256;
  EIG_TRY(h->small.reserve(sm));
  unsigned char* p = (unsigned char*)h->small.p;
  auto take = [&](size_t b) { unsigned char* r = p; p += (b + 255) & ~size_t(255); return r; };
  double* T = (double*)take((size_t)kmax * kmax * 8);
  double* Tk = (double*)take((size_t)kmax * kmax * 8);
  double* Cc = (double*)take((size_t)(maxblocks + 1) * nb * nb * 8);
  double* M = (double*)take((size_t)(maxblocks + 1) * nb * nb * 8);
  double* Z = (double*)take((size_t)kmax * mz * 8);
  double* wv = (double*)take(256 * 8);
  double* est = (double*)take(256 * 8);
  double* estp = (double*)take(256 * 8);
  double* R = (double*)take((size_t)nb * nb * 8);
  double* Zb = (double*)take((size_t)kmax * nb * 8);   // one block of columns of Z at a restart
  void* work = take(small_syev_work_bytes(kmax, mz));
  void* gpart = take(gsz);
  EIG_CUDA_TRY(cudaMemsetAsync(T, 0, (size_t)kmax * kmax * 8, c.st));
  // V_1 = orthonormal basis of X0 (Alg. 1 line 1)
  {
    DevBuf x64;
    EIG_TRY(x64.reserve((size_t)n * nb * 8));
    if (x0c >= nb) {
      EIG_TRY(pad_columns(X0, x0c, x64.as<double>(), nb, n, c.st));
    } else {
      // fewer guesses than the block: seeded random vectors fill the remaining columns
      EIG_TRY(fill_random(x64.as<double>(), n * nb, c.o.seed + 7, c.st));
      EIG_TRY(overlay_columns(X0, x0c, x64.as<double>(), nb, n, c.st));
    }
    EIG_TRY(convert(x64.p, EIG_F64, V[0], vt, n * nb, c.st));
    EIG_TRY(c.sync());
  }
  EIG_TRY(cholqr2_impl2(V[0], nullptr, n, nb, vt, R, c.st));
  EIG_TRY(h->host.reserve(256 * 8));
  double* hs = h->host.as<double>();
  std::vector<double> th(nev, 0.0), rel(nev, 0.0);
  *converged = false;
  *reason = 0;
  int it = -1, nblocks = 1, kdim = nb, restart_at = -1;
  for (int i = 0;; ++i) {
    ++it;
    // H V_i and CGS2 against the basis (Eq. bgs)
    EIG_TRY(c.spmm(V[i], HV, nb, vt, nb));
    EIG_TRY(basis_gram(c, V.data(), i + 1, HV, nb, vt, Cc, gpart));
    if (i == restart_at) {
      // first block after a thick restart: H Y = Y Theta + V_q S, so T's kept rows couple to it
      k_put_coupling<<<4, 256, 0, c.st>>>(T, kmax, i, nb, Cc);
      EIG_LAUNCH_CHECK("k_put_coupling");
    }
    k_put_blocks<<<1, 256, 0, c.st>>>(T, kmax, i, nb, Cc + (size_t)i * nb * nb, nullptr);
    EIG_LAUNCH_CHECK("k_put_blocks");
    {
      k_negate_stack<<<4, 256, 0, c.st>>>(Cc, i + 1, nb, M);
      EIG_LAUNCH_CHECK("k_negate_stack");
      BlockList in;
      in.n = i + 2;
      for (int b = 0; b <= i; ++b) in.p[b] = V[b];
      in.p[i + 1] = HV;
      EIG_TRY(block_apply(in, nb, M, nb, W, 0.0, n, vt, c.st));
      EIG_TRY(basis_gram(c, V.data(), i + 1, W, nb, vt, Cc, gpart));
      k_negate_stack<<<4, 256, 0, c.st>>>(Cc, i + 1, nb, M);
      EIG_LAUNCH_CHECK("k_negate_stack");
      in.p[i + 1] = W;
      EIG_TRY(block_apply(in, nb, M, nb, HV, 0.0, n, vt, c.st));  // HV now holds W_i
    }
    kdim = (i + 1) * nb;
    nblocks = i + 1;
    // QR of W_i: V_{i+1} R_{i+1} (R needed for the residual estimate)
    bool qr_ok = true;
    if (i + 1 <= maxblocks - 1 || true) {
      EIG_CUDA_TRY(cudaMemcpyAsync(V[std::min(i + 1, maxblocks)], HV, blk, cudaMemcpyDeviceToDevice, c.st));
      eig_status q = cholqr2_impl2(V[std::min(i + 1, maxblocks)], nullptr, n, nb, vt, R, c.st);
      if (q == EIG_EBREAKDOWN) {
        qr_ok = false;
        EIG_CUDA_TRY(cudaMemsetAsync(R, 0, (size_t)nb * nb * 8, c.st));
      } else if (q != EIG_OK) {
        return q;
      }
    }
    // projected problem T_{i+1} (Alg. 1 line 12-13)
    k_copy_lead<<<4, 256, 0, c.st>>>(T, kmax, kdim, Tk);
    EIG_LAUNCH_CHECK("k_copy_lead");
    const int m = std::min(nev, kdim);
    EIG_TRY(small_syev(Tk, kdim, m, wv, Z, work, nullptr, c.st));
    // residual estimate (exact form of Eq. ritzest2)
    double wf = 0.0;
    k_block_est<<<1, 64, 0, c.st>>>(R, Z, kdim, nb, m, wv, est, estp, wf);
    EIG_LAUNCH_CHECK("k_block_est");
    EIG_CUDA_TRY(cudaMemcpyAsync(hs, wv, m * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs + 64, est, m * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    bool conv = (m == nev);
    for (int t = 0; t < m; ++t) {
      th[t] = hs[t];
      rel[t] = hs[64 + t];
      conv = conv && rel[t] < c.o.tol;
    }
    c.trace(0, it, th.data(), rel.data(), m);
    if (conv) { *converged = true; break; }
    if (!qr_ok) { *reason = 4; break; }
    if (it >= maxiter) break;
    if (stop) {
      const int r = stop(it + 1, th.data(), rel.data(), m);
      if (r) { *reason = r; break; }
    }
    if (i + 1 >= maxblocks) {
      if (keep == 0) break;   // no restart: stop at the basis limit
      // thick restart (Sec. 2.2): Y = V Z(:, 1:keep) replaces the basis, V_{i+1} follows it,
      // T = diag(theta_1..keep) until the next block's Gram adds the couplings
      EIG_TRY(small_syev(Tk, kdim, keep, wv, Z, work, nullptr, c.st));
      BlockList in;
      in.n = i + 1;
      for (int b = 0; b <= i; ++b) in.p[b] = V[b];
      for (int b = 0; b < qkeep; ++b) {
        EIG_CUDA_TRY(cudaMemcpy2DAsync(Zb, nb * 8, Z + b * nb, (size_t)keep * 8, nb * 8, kdim,
                                       cudaMemcpyDeviceToDevice, c.st));
        EIG_TRY(block_apply(in, nb, Zb, nb, Ytmp + (size_t)b * blk, 0.0, n, vt, c.st));
      }
      for (int b = 0; b < qkeep; ++b)
        EIG_CUDA_TRY(cudaMemcpyAsync(V[b], Ytmp + (size_t)b * blk, blk, cudaMemcpyDeviceToDevice, c.st));
      EIG_CUDA_TRY(cudaMemcpyAsync(V[qkeep], V[i + 1], blk, cudaMemcpyDeviceToDevice, c.st));
      EIG_CUDA_TRY(cudaMemsetAsync(T, 0, (size_t)kmax * kmax * 8, c.st));
      k_set_diag<<<1, 256, 0, c.st>>>(T, kmax, wv, keep);
      EIG_LAUNCH_CHECK("k_set_diag");
      restart_at = qkeep;
      i = qkeep - 1;
      continue;
    }
    // append R_{i+1} to T
    k_put_blocks<<<1, 256, 0, c.st>>>(T, kmax, i, nb, nullptr, R);
    EIG_LAUNCH_CHECK("k_put_blocks");
  }
  *iters = it;
  // X = V Z (Alg. 1 "X_{i+1} = V U(:, 1:nev)")
  EIG_TRY(h->Xres.reserve((size_t)n * nev * 8));
  {
    DevBuf Xt;
    EIG_TRY(Xt.reserve((size_t)n * nev * sv));
    BlockList in;
    in.n = nblocks;
    for (int b = 0; b < nblocks; ++b) in.p[b] = V[b];
    EIG_TRY(block_apply(in, nb, Z, nev, Xt.p, 0.0, n, vt, c.st));
    EIG_TRY(convert(Xt.p, vt, h->Xres.p, EIG_F64, n * nev, c.st));
    EIG_TRY(c.sync());
  }
  theta_out->assign(th.begin(), th.end());
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// ChebFSI (Alg. 3)
// ---------------------------------------------------------------------------------------
eig_status run_chebfsi(Ctx& c, const double* X0, int x0c, int* iters, bool* converged,
                       std::vector<double>* theta_out) {
  Handle* h = c.h;
  const int nb = h->nb, nev = h->n_ev;
  const int64_t n = h->n;
  const eig_dtype vt = c.o.vec_type;
  const size_t sv = dtype_size(vt);
  const int deg = std::max(1, c.o.cheb_degree);
  double lub = c.o.lambda_ub;
  if (!(lub > 0.0) && !(lub < 0.0)) {
    EIG_TRY(lambda_ub_estimate(c, 10, &lub));
    c.s->spmv_count += 10;
  }
  for (int b = 0; b < 6; ++b) EIG_TRY(h->blk[b].reserve((size_t)n * nb * sv));
  void *Q = h->blk[0].p, *HQ = h->blk[1].p, *Wb = h->blk[2].p, *Qp = h->blk[3].p, *Y = h->blk[4].p,
       *HW = h->blk[5].p;
  const size_t gsz = gram_scratch_bytes(1, nb);
  EIG_TRY(h->small.reserve((size_t)nb * nb * 8 * 4 + 64 * 8 * 4 + small_syev_work_bytes(nb, nb) + gsz +
                           colsum_scratch_bytes(nb) + 16 * 256 + (size_t)num_sms() * 8 * nb * 8));
  unsigned char* p = (unsigned char*)h->small.p;
  auto take = [&](size_t b) { unsigned char* r = p; p += (b + 255) & ~size_t(255); return r; };
  double* Tm = (double*)take((size_t)nb * nb * 8);
  double* S = (double*)take((size_t)nb * nb * 8);
  double* R = (double*)take((size_t)nb * nb * 8);
  double* th_d = (double*)take(64 * 8);
  double* rs = (double*)take(64 * 8);
  double* nrm = (double*)take(64 * 8);
  int* act_d = (int*)take(64 * 4);
  void* work = take(small_syev_work_bytes(nb, nb));
  void* gpart = take(gsz);
  void* cpart = take(colsum_scratch_bytes(nb));
  double* rpart = (double*)take((size_t)num_sms() * 8 * nb * 8);
  EIG_TRY(h->host.reserve(256 * 8));
  double* hs = h->host.as<double>();
  // Q = CholeskyQR(X0) (Alg. 3 line 3)
  {
    DevBuf x64;
    EIG_TRY(x64.reserve((size_t)n * nb * 8));
    if (x0c >= nb) {
      EIG_TRY(pad_columns(X0, x0c, x64.as<double>(), nb, n, c.st));
    } else {
      EIG_TRY(fill_random(x64.as<double>(), n * nb, c.o.seed + 7, c.st));
      EIG_TRY(overlay_columns(X0, x0c, x64.as<double>(), nb, n, c.st));
    }
    EIG_TRY(convert(x64.p, EIG_F64, Q, vt, n * nb, c.st));
    EIG_TRY(c.sync());
  }
  EIG_TRY(cholqr2_impl2(Q, nullptr, n, nb, vt, R, c.st));
  EIG_TRY(c.spmm(Q, HQ, nb, vt, nb));
  const int rgrid = num_sms() * 8;
  const int rthreads = (256 / nb) * nb;
  auto rayleigh_ritz = [&]() -> eig_status {
    BlockList bl;
    bl.n = 2;
    bl.p[0] = Q;
    bl.p[1] = HQ;
    const int pa = 0, pb = 1;
    EIG_TRY(gram_multi(bl, &pa, &pb, 1, nb, n, vt, Tm, gpart, c.st));
    EIG_TRY(small_syev(Tm, nb, nb, th_d, S, work, nullptr, c.st));
    BlockList in;
    in.n = 1;
    in.p[0] = Q;
    EIG_TRY(block_apply(in, nb, S, nb, Y, 0.0, n, vt, c.st));
    in.p[0] = HQ;
    EIG_TRY(block_apply(in, nb, S, nb, HW, 0.0, n, vt, c.st));
    std::swap(Q, Y);
    std::swap(HQ, HW);
    if (vt == EIG_F32) k_resid_sumsq<float><<<rgrid, rthreads, 0, c.st>>>((const float*)Q, (const float*)HQ, th_d, nb, n, rpart);
    else k_resid_sumsq<double><<<rgrid, rthreads, 0, c.st>>>((const double*)Q, (const double*)HQ, th_d, nb, n, rpart);
    EIG_LAUNCH_CHECK("k_resid_sumsq");
    EIG_TRY(reduce_partials(rpart, rgrid, nb, rs, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs, th_d, nb * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs + 64, rs, nb * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    return EIG_OK;
  };
  EIG_TRY(rayleigh_ritz());
  std::vector<double> th(nb), rel(nb);
  std::vector<int> act(nb);
  auto status = [&]() {
    bool conv = true;
    for (int j = 0; j < nb; ++j) {
      th[j] = hs[j];
      rel[j] = std::sqrt(std::max(hs[64 + j], 0.0)) / std::max(std::fabs(th[j]), 1e-300);
      act[j] = rel[j] < c.o.tol ? 0 : 1;
      if (j < nev) conv = conv && rel[j] < c.o.tol;
    }
    return conv;
  };
  bool conv = status();
  c.trace(0, 0, th.data(), rel.data(), nev);
  int it = 0;
  while (!conv && it < c.o.maxiter) {
    ++it;
    const double lf = th[nb - 1];
    const double cc = 0.5 * (lub + lf), ee = 0.5 * (lub - lf);
    int nact = 0;
    for (int j = 0; j < nb; ++j) nact += act[j];
    EIG_CUDA_TRY(cudaMemcpyAsync(act_d, act.data(), nb * 4, cudaMemcpyHostToDevice, c.st));
    const int g = num_sms() * 8;
    // W = (HQ - cQ)/e ; Qp = Q
    EIG_CUDA_TRY(cudaMemcpyAsync(Qp, Q, (size_t)n * nb * sv, cudaMemcpyDeviceToDevice, c.st));
    if (vt == EIG_F32) k_cheb<float><<<g, 256, 0, c.st>>>((const float*)HQ, (const float*)Q, nullptr, (float*)Wb, act_d, cc, ee, 1, nb, n);
    else k_cheb<double><<<g, 256, 0, c.st>>>((const double*)HQ, (const double*)Q, nullptr, (double*)Wb, act_d, cc, ee, 1, nb, n);
    EIG_LAUNCH_CHECK("k_cheb");
    for (int j = 2; j <= deg; ++j) {
      // Y = 2 (H W - c W) / e - Qp: fused into the SpMM's epilogue where the layout allows it
      // (one read of W and Qp, one write of Y), else the product then the elementwise step
      const eig_status fs = c.spmm_cheb(Wb, Y, nb, vt, nact, Qp, act_d, 2.0 / ee, cc, 0);
      if (fs == EIG_EUNSUPPORTED) {
        EIG_TRY(c.spmm(Wb, HW, nb, vt, nact));
        if (vt == EIG_F32) k_cheb<float><<<g, 256, 0, c.st>>>((const float*)HW, (const float*)Wb, (const float*)Qp, (float*)Y, act_d, cc, ee, 0, nb, n);
        else k_cheb<double><<<g, 256, 0, c.st>>>((const double*)HW, (const double*)Wb, (const double*)Qp, (double*)Y, act_d, cc, ee, 0, nb, n);
        EIG_LAUNCH_CHECK("k_cheb");
      } else {
        EIG_TRY(fs);
      }
      std::swap(Qp, Wb);  // Qp <- W
      std::swap(Wb, Y);   // W <- Y
    }
    // Wb holds T_d(...) Q; HW <- H Wb (locked columns: H Q unchanged up to rounding)
    EIG_TRY(c.spmm(Wb, HW, nb, vt, nact));
    // unit columns, then CholQR2 with the same transform applied to H W (so HQ = HY R^{-1})
    EIG_TRY(col_sumsq(Wb, nb, n, vt, nrm, cpart, c.st));
    if (vt == EIG_F32) k_scale_cols<float><<<g, 256, 0, c.st>>>((float*)Wb, (float*)HW, nrm, nb, n);
    else k_scale_cols<double><<<g, 256, 0, c.st>>>((double*)Wb, (double*)HW, nrm, nb, n);
    EIG_LAUNCH_CHECK("k_scale_cols");
    EIG_TRY(cholqr2_impl2(Wb, HW, n, nb, vt, R, c.st));
    std::swap(Q, Wb);
    std::swap(HQ, HW);
    EIG_TRY(rayleigh_ritz());
    conv = status();
    c.trace(0, it, th.data(), rel.data(), nev);
  }
  *iters = it;
  *converged = conv;
  EIG_TRY(h->Xres.reserve((size_t)n * nev * 8));
  {
    DevBuf X64;
    EIG_TRY(X64.reserve((size_t)n * nb * 8));
    EIG_TRY(convert(Q, vt, X64.p, EIG_F64, n * nb, c.st));
    EIG_TRY(pad_columns(X64.as<double>(), nb, h->Xres.as<double>(), nev, n, c.st));
    EIG_TRY(c.sync());
  }
  // keep the handle's block pointers consistent with the swapped roles
  h->blk[0].p = Q; h->blk[1].p = HQ; h->blk[2].p = Wb; h->blk[3].p = Qp; h->blk[4].p = Y; h->blk[5].p = HW;
  theta_out->assign(th.begin(), th.begin() + nev);
  return EIG_OK;
}

}  // namespace eig
