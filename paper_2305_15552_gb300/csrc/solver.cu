// Solver drivers: LOBPCG (Alg. 2), batched RMM-DIIS (Alg. 4, Sec. 4.3) and the hybrid of
// Sec. 4, plus the eig_create / eig_solve / eig_ritz C ABI.
//
// Control stays on the host: each iteration enqueues its kernels on the caller's stream and
// reads back one small status record (Ritz values and residual norms) to decide convergence
// and the switch of Eq. (switchtau).  All arithmetic runs in this library's kernels.
#include <algorithm>
#include <cmath>
#include <new>

#include "common.cuh"
#include "dense.cuh"
#include "rmm.cuh"
#include "small.cuh"
#include "solver.cuh"
#include "learned.cuh"
#include "spmm.cuh"

namespace eig {

// ---------------------------------------------------------------------------------------
// helper kernels
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_fill_random(double* X, int64_t count, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = splitmix64(seed * 0x9E3779B97F4A7C15ull ^ (uint64_t)i);
    X[i] = (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

eig_status fill_random(double* X, int64_t count, uint64_t seed, cudaStream_t st) {
  k_fill_random<<<num_sms() * 4, 256, 0, st>>>(X, count, seed);
  EIG_LAUNCH_CHECK("k_fill_random");
  return EIG_OK;
}

__global__ void k_pad_columns(const double* __restrict__ src, int ks, double* __restrict__ dst, int kd, int64_t n) {
  const int64_t total = n * kd;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kd;
    const int j = (int)(i % kd);
    dst[i] = (j < ks) ? src[r * ks + j] : 0.0;
  }
}

// y += a x over count entries
__global__ void k_add_scaled(const double* __restrict__ x, double a, double* __restrict__ y, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

eig_status pad_columns(const double* src, int ks, double* dst, int kd, int64_t n, cudaStream_t st) {
  k_pad_columns<<<num_sms() * 8, 256, 0, st>>>(src, ks, dst, kd, n);
  EIG_LAUNCH_CHECK("k_pad_columns");
  return EIG_OK;
}

// per-column partial dots of two FP64 blocks (n x m), and residual norms ||hx - theta x||^2
__global__ void k_coldot2(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ theta,
                          int m, int64_t n, double* __restrict__ part) {
  __shared__ double red[256 * 2];
  const int j = threadIdx.x % m, rr = threadIdx.x / m, rpp = blockDim.x / m;
  double v0 = 0.0, v1 = 0.0;
  const double th = theta ? theta[j] : 0.0;
  if (rr < rpp) {
    for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
      const double x = a[r * m + j], h = b[r * m + j];
      v0 = fma(x, h, v0);
      const double res = h - th * x;
      v1 = fma(res, res, v1);
    }
  }
  red[threadIdx.x * 2] = (rr < rpp) ? v0 : 0.0;
  red[threadIdx.x * 2 + 1] = (rr < rpp) ? v1 : 0.0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < m * 2; idx += blockDim.x) {
    const int jj = idx / 2, q = idx % 2;
    double s = 0.0;
    for (int r2 = 0; r2 < rpp; ++r2) s += red[(r2 * m + jj) * 2 + q];
    part[((size_t)blockIdx.x * m + jj) * 2 + q] = s;
  }
}

// Assemble full symmetric k x k matrices from block pair products: pairs (a, b), a <= b.
struct PairMap {
  int idx[4][4];  // pair index for (a, b), -1 if absent
};
__global__ void k_assemble(const double* __restrict__ Gp, PairMap map, int nblk, int nb, double* __restrict__ out) {
  const int k = nblk * nb;
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < k * k; e += blockDim.x * gridDim.x) {
    const int row = e / k, col = e % k;
    const int a = row / nb, i = row % nb, b = col / nb, j = col % nb;
    double v;
    if (a <= b) v = Gp[(size_t)map.idx[a][b] * nb * nb + i * nb + j];
    else v = Gp[(size_t)map.idx[b][a] * nb * nb + j * nb + i];
    out[e] = v;
  }
}

__global__ void k_pack_rmm_dots(const double* __restrict__ sc, const double* __restrict__ s4, int mp,
                                int preconditioned, double* __restrict__ dots) {
  const int j = threadIdx.x;
  if (j >= mp) return;
  // dots: <x,x>, <x,Hx>, <x,r>, <r,r>, <x,Hr>, <r,Hr>; sc = combine sums (stride 5), s4 = dots4 sums.
  // The off-diagonal of W^T H W is symmetrised, (<x,Hr> + <r,Hx>)/2 (H x~ comes from the history
  // by linearity, H r~ from the SpMM).
  dots[j * 6 + 0] = sc[j * 5 + 0];
  dots[j * 6 + 1] = sc[j * 5 + 1];
  dots[j * 6 + 2] = s4[j * 4 + 2];
  dots[j * 6 + 3] = s4[j * 4 + 3];
  dots[j * 6 + 4] = 0.5 * (s4[j * 4 + 0] + (preconditioned ? s4[j * 4 + 0] : sc[j * 5 + 4]));
  dots[j * 6 + 5] = s4[j * 4 + 1];
}

// x~/r~ dots after an optional preconditioning of r~: <x~,Hr~>, <r~,Hr~>, <x~,r~>, <r~,r~>
template <typename T>
__global__ void k_rmm_dots4(const double* __restrict__ xt, const T* __restrict__ rt, const T* __restrict__ hrt, int mp,
                            int64_t n, double* __restrict__ part) {
  __shared__ double red[256 * 4];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  double v[4] = {0, 0, 0, 0};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const double x = xt[e], rv = (double)rt[e], h = (double)hrt[e];
    v[0] = fma(x, h, v[0]);
    v[1] = fma(rv, h, v[1]);
    v[2] = fma(x, rv, v[2]);
    v[3] = fma(rv, rv, v[3]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[threadIdx.x * 4 + q] = v[q];
  __syncthreads();
  for (int idx = threadIdx.x; idx < mp * 4; idx += blockDim.x) {
    const int jj = idx / 4, q = idx % 4;
    double s = 0.0;
    for (int r2 = 0; r2 < rpp; ++r2) s += red[(r2 * mp + jj) * 4 + q];
    part[((size_t)blockIdx.x * mp + jj) * 4 + q] = s;
  }
}

__global__ void k_overlay_columns(const double* __restrict__ src, int ks, double* __restrict__ dst, int kd,
                                  int64_t n) {
  const int64_t total = n * ks;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ks;
    const int j = (int)(i % ks);
    if (j < kd) dst[r * kd + j] = src[i];
  }
}

eig_status overlay_columns(const double* src, int ks, double* dst, int kd, int64_t n, cudaStream_t st) {
  k_overlay_columns<<<num_sms() * 8, 256, 0, st>>>(src, ks, dst, kd, n);
  EIG_LAUNCH_CHECK("k_overlay_columns");
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------------------
static int spmm_shape_index(int nb, eig_dtype vt) {
  int l = 0;
  while ((1 << l) < nb && l < 5) ++l;
  return 6 * (vt == EIG_F64 ? 1 : 0) + l;
}

void Ctx::count_spmm(int nb, eig_dtype vt, int64_t spmv_cols) {
  const double bytes = h->plan.algorithmic_bytes(nb, dtype_size(vt));
  const int k = spmm_shape_index(nb, vt);
  s->spmm_calls += 1;
  s->spmv_count += spmv_cols;
  s->spmm_bytes += bytes;
  s->spmm_calls_by_shape[k] += 1;
  s->spmm_bytes_by_shape[k] += bytes;
  if (o.timing) spmm_shape.push_back(k);
}

eig_status Ctx::spmm(const void* X, void* Y, int nb, eig_dtype vt, int64_t spmv_cols) {
  if (batch) {
    SpmmJob j{&h->plan, X, Y, nullptr, nullptr, 0.0, 0.0, 0};
    EIG_TRY(batch_product(batch, *this, j, nb, vt, false));
    count_spmm(nb, vt, spmv_cols);
    return EIG_OK;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (o.timing) {
    EIG_CUDA_TRY(cudaEventCreate(&a));
    EIG_CUDA_TRY(cudaEventCreate(&b));
    EIG_CUDA_TRY(cudaEventRecord(a, st));
  }
  EIG_TRY(spmm_run(&h->plan, X, Y, nb, vt, st));
  if (o.timing) {
    EIG_CUDA_TRY(cudaEventRecord(b, st));
    spmm_ev.emplace_back(a, b);
  }
  count_spmm(nb, vt, spmv_cols);
  return EIG_OK;
}

eig_status Ctx::spmv_col(const void* X, void* Y, int ld, int col, eig_dtype vt) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (o.timing) {
    EIG_CUDA_TRY(cudaEventCreate(&a));
    EIG_CUDA_TRY(cudaEventCreate(&b));
    EIG_CUDA_TRY(cudaEventRecord(a, st));
  }
  const eig_status r = spmm_run_column(&h->plan, X, Y, ld, col, vt, st);
  if (r != EIG_OK) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return r;
  }
  if (o.timing) {
    EIG_CUDA_TRY(cudaEventRecord(b, st));
    spmm_ev.emplace_back(a, b);
  }
  count_spmm(1, vt, 1);
  return EIG_OK;
}

eig_status Ctx::rmm_product(const void* X, void* Y, int mp, eig_dtype vt, const std::vector<int>& act, int nev) {
  int nact = 0;
  for (int j = 0; j < mp; ++j) nact += act[j];
  if (o.rmm_decouple > 0 && nev - nact >= o.rmm_decouple && h->plan.mirrored) {
    for (int j = 0; j < mp; ++j)
      if (act[j]) EIG_TRY(spmv_col(X, Y, mp, j, vt));
    return EIG_OK;
  }
  return spmm(X, Y, mp, vt, nact);
}

eig_status Ctx::spmm_cheb(const void* X, void* Y, int nb, eig_dtype vt, int64_t spmv_cols, const void* Qp,
                          const int* active, double alpha, double cshift, int first) {
  if (batch) {
    if (!h->plan.mirrored || (nb != 8 && nb != 16 && nb != 32)) return EIG_EUNSUPPORTED;
    SpmmJob j{&h->plan, X, Y, Qp, active, alpha, cshift, first};
    EIG_TRY(batch_product(batch, *this, j, nb, vt, true));
    count_spmm(nb, vt, spmv_cols);
    return EIG_OK;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (o.timing) {
    EIG_CUDA_TRY(cudaEventCreate(&a));
    EIG_CUDA_TRY(cudaEventCreate(&b));
    EIG_CUDA_TRY(cudaEventRecord(a, st));
  }
  const eig_status r = spmm_run_cheb(&h->plan, X, Y, nb, vt, Qp, active, alpha, cshift, first, st);
  if (r != EIG_OK) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return r;
  }
  if (o.timing) {
    EIG_CUDA_TRY(cudaEventRecord(b, st));
    spmm_ev.emplace_back(a, b);
  }
  count_spmm(nb, vt, spmv_cols);
  return EIG_OK;
}

Ctx::~Ctx() {
  for (auto& e : spmm_ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (req_ev) cudaEventDestroy(req_ev);
}

// Small-workspace carving
struct Carve {
  unsigned char* base;
  size_t off = 0, cap;
  Carve(void* p, size_t c) : base((unsigned char*)p), cap(c) {}
  template <typename T> T* take(size_t count) {
    size_t b = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + b > cap) {  // sizing error: callers check ok() before any launch
      bad = true;
      return nullptr;
    }
    T* r = (T*)(base + off);
    off += b;
    return r;
  }
  bool ok() const { return !bad; }
  bool bad = false;
};

// Learned K^{-1} (precond / rmm_precond = 2) on the residual block R (n x ld, first m columns),
// written to W (may alias R): one SpMM for H R into HR (scratch), then the fused feature + MLP
// kernel.  theta, rsq: device FP64 [m]; active may be null.
static eig_status lp_precondition(Ctx& c, const void* R, void* HR, int ld, int m, eig_dtype vt, const double* theta,
                                  const double* rsq, const int* active, int64_t spmv_cols, void* W, int* nonfinite) {
  Handle* h = c.h;
  EIG_TRY(lp_ensure_rowabs(h, c.st));
  EIG_TRY(c.spmm(R, HR, ld, vt, spmv_cols));
  c.s->lp_spmm_calls += 1;
  LpParams prm;
  std::memcpy(prm.p, c.o.lp_params, sizeof(prm.p));
  return lp_apply(prm, R, HR, ld, m, h->n, vt, h->plan.diag.as<double>(), h->lp_rowabs.as<double>(), theta, rsq,
                  c.o.precond_floor, active, W, nonfinite, c.st);
}

// ---------------------------------------------------------------------------------------
// certification: true FP64 residuals of (theta_j, x_j) for the returned pairs
// ---------------------------------------------------------------------------------------
// Gram of the first m columns of X (n x ld, FP64) for the duplicate check: the m(m+1)/2 pairs
// are spread over the CTA's threads (sets of `npairs` threads take interleaved rows), FP64 sums,
// fixed-order reductions.  part: [cta][npairs].
__global__ void k_pair_gram(const double* __restrict__ X, int m, int ld, int64_t n, double* __restrict__ part) {
  __shared__ double red[256];
  const int npairs = m * (m + 1) / 2;
  const int sets = blockDim.x / npairs;
  const int p = threadIdx.x % npairs, set = threadIdx.x / npairs;
  int i = 0, j = p;
  while (j >= m - i) { j -= m - i; ++i; }
  j += i;
  double acc = 0.0;
  if (set < sets)
    for (int64_t r = blockIdx.x * (int64_t)sets + set; r < n; r += (int64_t)gridDim.x * sets)
      acc = fma(X[r * ld + i], X[r * ld + j], acc);
  red[threadIdx.x] = (set < sets) ? acc : 0.0;
  __syncthreads();
  if (threadIdx.x < npairs) {
    double t = 0.0;
    for (int q = 0; q < sets; ++q) t += red[q * npairs + threadIdx.x];
    part[(size_t)blockIdx.x * npairs + threadIdx.x] = t;
  }
}

// Two columns of X (n x ld, FP64, first m used) that are collinear (|cos| >= 0.9) with Ritz values
// equal to 1e-6 relative: RMM-DIIS does not orthogonalise its vectors (Sec. 3.3).
// Symmetric Gram matrix hg (ld x ld, host) of the first m columns of X (n x ld, FP64).
static eig_status column_gram(Ctx& c, const double* X, int m, int ld, std::vector<double>* hg) {
  const int npairs = m * (m + 1) / 2;
  const int grid = num_sms() * 4;
  DevBuf gbuf;
  EIG_TRY(gbuf.reserve((size_t)grid * npairs * 8 + (size_t)npairs * 8));
  double* part = gbuf.as<double>();
  double* Gp = part + (size_t)grid * npairs;
  k_pair_gram<<<grid, 256, 0, c.st>>>(X, m, ld, c.h->n, part);
  EIG_LAUNCH_CHECK("k_pair_gram");
  EIG_TRY(reduce_partials(part, grid, npairs, Gp, c.st));
  std::vector<double> hp(npairs);
  hg->assign((size_t)ld * ld, 0.0);
  EIG_CUDA_TRY(cudaMemcpyAsync(hp.data(), Gp, npairs * 8, cudaMemcpyDeviceToHost, c.st));
  EIG_TRY(c.sync());
  for (int i = 0, q = 0; i < m; ++i)
    for (int j = i; j < m; ++j, ++q) (*hg)[(size_t)i * ld + j] = (*hg)[(size_t)j * ld + i] = hp[q];
  return EIG_OK;
}

eig_status find_duplicates(Ctx& c, const double* X, int m, int ld, const std::vector<double>& theta,
                           bool* duplicate) {
  *duplicate = false;
  if (m < 2) return EIG_OK;
  if (m * (m + 1) / 2 > 256) return EIG_OK;  // n_ev > 22: no check
  std::vector<double> hg;
  EIG_TRY(column_gram(c, X, m, ld, &hg));
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double gi = hg[(size_t)i * ld + i], gj = hg[(size_t)j * ld + j];
      const double cosv = std::fabs(hg[(size_t)i * ld + j]) / std::sqrt(std::max(gi * gj, 1e-300));
      const double scale = std::max(std::max(std::fabs(theta[i]), std::fabs(theta[j])), 1e-300);
      if (cosv >= 0.9 && std::fabs(theta[i] - theta[j]) <= 1e-6 * scale) *duplicate = true;
    }
  return EIG_OK;
}

// Columns of X (n x ld, first m) to keep as a start block: in order, a column is dropped when
// |cos| with a kept one is >= cos_max (RMM-DIIS can leave several on one eigenvector).
static eig_status independent_columns(Ctx& c, const double* X, int m, int ld, double cos_max, std::vector<int>* keep) {
  keep->clear();
  if (m * (m + 1) / 2 > 256) {
    for (int j = 0; j < m; ++j) keep->push_back(j);
    return EIG_OK;
  }
  std::vector<double> hg;
  EIG_TRY(column_gram(c, X, m, ld, &hg));
  for (int j = 0; j < m; ++j) {
    const double gj = hg[(size_t)j * ld + j];
    bool ok = gj > 0.0;
    for (int i : *keep) {
      const double gi = hg[(size_t)i * ld + i];
      if (std::fabs(hg[(size_t)i * ld + j]) >= cos_max * std::sqrt(gi * gj)) ok = false;
    }
    if (ok) keep->push_back(j);
  }
  return EIG_OK;
}

struct ColIdx {
  int c[32];
};

// dst (n x kd) column q <- src (n x ks) column idx.c[q]
__global__ void k_gather_columns(const double* __restrict__ src, int ks, ColIdx idx, int kd, double* __restrict__ dst,
                                 int64_t n) {
  const int64_t total = n * kd;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / kd;
    dst[i] = src[r * ks + idx.c[i % kd]];
  }
}

// Also flags duplicates: two returned vectors that are collinear (|cos| >= 0.9) with Ritz values
// equal to 1e-6 relative (RMM-DIIS does not orthogonalise its vectors, Sec. 3.3).
eig_status certify(Ctx& c, const double* X, const std::vector<double>& theta, std::vector<double>* relres,
                   bool* duplicate) {
  Handle* h = c.h;
  const int m = h->n_ev, mp = next_pow2(m);
  const int64_t n = h->n;
  EIG_TRY(h->tmp64a.reserve((size_t)n * mp * 8));
  EIG_TRY(h->tmp64b.reserve((size_t)n * mp * 8));
  double* Xp = h->tmp64a.as<double>();
  double* HXp = h->tmp64b.as<double>();
  EIG_TRY(pad_columns(X, m, Xp, mp, n, c.st));
  EIG_TRY(spmm_run(&h->plan, Xp, HXp, mp, EIG_F64, c.st));
  const int grid = num_sms() * 4;
  DevBuf tmp;
  EIG_TRY(tmp.reserve((size_t)grid * mp * 2 * 8 + mp * 2 * 8 + mp * 8));
  double* part = tmp.as<double>();
  double* sums = part + (size_t)grid * mp * 2;
  double* th = sums + mp * 2;
  std::vector<double> thp(mp, 0.0);
  for (int j = 0; j < m; ++j) thp[j] = theta[j];
  EIG_CUDA_TRY(cudaMemcpyAsync(th, thp.data(), mp * 8, cudaMemcpyHostToDevice, c.st));
  const int threads = (256 / mp) * mp;
  k_coldot2<<<grid, threads, 0, c.st>>>(Xp, HXp, th, mp, n, part);
  EIG_LAUNCH_CHECK("k_coldot2");
  EIG_TRY(reduce_partials(part, grid, mp * 2, sums, c.st));
  std::vector<double> hs(mp * 2);
  EIG_CUDA_TRY(cudaMemcpyAsync(hs.data(), sums, mp * 2 * 8, cudaMemcpyDeviceToHost, c.st));
  // column norms of X
  EIG_TRY(col_sumsq(Xp, mp, n, EIG_F64, sums, part, c.st));
  std::vector<double> nn(mp);
  EIG_CUDA_TRY(cudaMemcpyAsync(nn.data(), sums, mp * 8, cudaMemcpyDeviceToHost, c.st));
  EIG_TRY(c.sync());
  relres->assign(m, 0.0);
  for (int j = 0; j < m; ++j) {
    const double xn = std::sqrt(std::max(nn[j], 1e-300));
    (*relres)[j] = std::sqrt(std::max(hs[j * 2 + 1], 0.0)) / xn / std::max(std::fabs(theta[j]), 1e-300);
  }
  EIG_TRY(find_duplicates(c, Xp, m, mp, theta, duplicate));
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// LOBPCG (Alg. 2)
// ---------------------------------------------------------------------------------------
eig_status run_lobpcg(Ctx& c, const double* X0, int x0_cols, int maxiter, const StopFn& stop, int* iters,
                      int* reason, bool* converged, double* X64_out, std::vector<double>* theta_out) {
  Handle* h = c.h;
  const int nb = h->nb, nev = h->n_ev;
  const int64_t n = h->n;
  const eig_dtype vt = c.o.vec_type;
  const size_t sv = dtype_size(vt);
  // squared pivots of the unit-diagonal Gram below this mark a basis too close to rank deficient
  // for the projected problem (cond > 1e5 in FP32, 1e10 in FP64): the pivoted path takes over
  const double piv_tol = (vt == EIG_F32) ? 1e-6 : 1e-10;
  for (int b = 0; b < 6; ++b) EIG_TRY(h->blk[b].reserve((size_t)n * nb * sv));
  void *X = h->blk[0].p, *W = h->blk[1].p, *P = h->blk[2].p, *HX = h->blk[3].p, *HW = h->blk[4].p, *HP = h->blk[5].p;
  const int kmax = 3 * nb;
  const int ugrid = update_grid(n);
  const size_t small_bytes = 12 * nb * nb * 8 + 2 * kmax * kmax * 8 + kmax * nb * 8 + kmax * nb * 4 + 64 * 8 +
                             small_rr_work_bytes(kmax, nb) + gram_scratch_bytes(12, nb) + (size_t)ugrid * nb * 8 +
                             32 * 256;
  EIG_TRY(h->small.reserve(small_bytes));
  Carve cv(h->small.p, h->small.bytes);
  double* Gp = cv.take<double>(12 * nb * nb);
  double* G = cv.take<double>(kmax * kmax);
  double* A = cv.take<double>(kmax * kmax);
  double* C = cv.take<double>(kmax * nb);
  double* stat = cv.take<double>(2 * nb + 8);  // theta[nb], rsq[nb], info
  int* info = reinterpret_cast<int*>(stat + 2 * nb);
  void* rrwork = cv.take<unsigned char>(small_rr_work_bytes(kmax, nb));
  void* gpart = cv.take<unsigned char>(gram_scratch_bytes(12, nb));
  double* upart = cv.take<double>((size_t)ugrid * nb);
  if (!cv.ok()) return EIG_EUNSUPPORTED;
  double* theta = stat;
  double* rsq = stat + nb;
  EIG_TRY(h->host.reserve((2 * nb + 8) * 8 + (size_t)kmax * nb * 8 + (size_t)kmax * kmax * 8));
  double* hstat = h->host.as<double>();
  const double* diagH = h->plan.diag.as<double>();
  // learned K^{-1} (precond = 2): the update forms plain residuals, lp_precondition scales them
  bool lp_on = c.o.precond == 2;
  if (lp_on && !c.o.lp_params) return EIG_EINVAL;
  auto upd_precond = [&]() { return lp_on ? 0 : (c.o.precond ? 1 : 0); };
  int* nonfin = reinterpret_cast<int*>(stat + 2 * nb + 1);
  EIG_CUDA_TRY(cudaMemsetAsync(nonfin, 0, 4, c.st));
  double lp_prev = 0.0;
  // X = X0 (FP64 n x x0_cols, x0_cols >= nb ... padded with random when fewer)
  EIG_TRY(h->tmp64a.reserve((size_t)n * nb * 8));
  double* X0p = h->tmp64a.as<double>();
  if (x0_cols < nb) {
    // fewer guesses than the block: the remaining columns start from seeded random vectors
    EIG_TRY(fill_random(X0p, n * nb, c.o.seed + 7, c.st));
    k_overlay_columns<<<num_sms() * 8, 256, 0, c.st>>>(X0, x0_cols, X0p, nb, n);
    EIG_LAUNCH_CHECK("k_overlay_columns");
  } else {
    EIG_TRY(pad_columns(X0, x0_cols, X0p, nb, n, c.st));  // the first nb columns
  }
  // initial Rayleigh-Ritz on X0 (Alg. 2 line 1)
  for (int attempt = 0;; ++attempt) {
    EIG_TRY(convert(X0p, EIG_F64, X, vt, n * nb, c.st));
    EIG_TRY(c.spmm(X, HX, nb, vt, nb));
    BlockList bl;
    bl.n = 2;
    bl.p[0] = X;
    bl.p[1] = HX;
    const int pa[2] = {0, 0}, pb[2] = {0, 1};
    EIG_TRY(gram_multi(bl, pa, pb, 2, nb, n, vt, Gp, gpart, c.st));
    PairMap mp;
    for (auto& r : mp.idx) for (int& v : r) v = -1;
    mp.idx[0][0] = 0;
    k_assemble<<<1, 256, 0, c.st>>>(Gp, mp, 1, nb, G);
    EIG_LAUNCH_CHECK("k_assemble");
    mp.idx[0][0] = 1;
    k_assemble<<<1, 256, 0, c.st>>>(Gp, mp, 1, nb, A);
    EIG_LAUNCH_CHECK("k_assemble");
    // a start block closer to rank deficiency than this is perturbed below rather than used
    EIG_TRY(small_rr(A, G, nb, nb, std::max(piv_tol, 1e-10), theta, C, nullptr, rrwork, info, c.st));
    BlockList in;
    in.n = 1;
    in.p[0] = X;
    EIG_TRY(block_apply(in, nb, C, nb, P, 0.0, n, vt, c.st));
    in.p[0] = HX;
    EIG_TRY(block_apply(in, nb, C, nb, HP, 0.0, n, vt, c.st));
    std::swap(h->blk[0].p, h->blk[2].p);
    std::swap(h->blk[3].p, h->blk[5].p);
    X = h->blk[0].p; P = h->blk[2].p; HX = h->blk[3].p; HP = h->blk[5].p;
    int np = 0;
    EIG_TRY(lobpcg_update(X, W, P, HX, HW, HP, C, nb, nb, theta, diagH, c.o.precond_floor, upd_precond(), n, vt,
                          upart, ugrid, &np, c.st));
    EIG_TRY(reduce_partials(upart, np, nb, rsq, c.st));
    if (lp_on) EIG_TRY(lp_precondition(c, W, HW, nb, nb, vt, theta, rsq, nullptr, nb, W, nonfin));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat, stat, (2 * nb + 8) * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    if (*reinterpret_cast<int*>(hstat + 2 * nb) == SMALL_OK) break;
    if (attempt == 2) return EIG_EBREAKDOWN;
    // the start block is numerically rank deficient (two guesses nearly parallel, as RMM-DIIS
    // can leave them): mix in a seeded random block of 1% of a unit column's norm and retry
    DevBuf rnd;
    EIG_TRY(rnd.reserve((size_t)n * nb * 8));
    EIG_TRY(fill_random(rnd.as<double>(), n * nb, c.o.seed + 1001 + attempt, c.st));
    k_add_scaled<<<num_sms() * 8, 256, 0, c.st>>>(rnd.as<double>(), 1e-2 / std::sqrt((double)n), X0p, n * nb);
    EIG_LAUNCH_CHECK("k_add_scaled");
  }
  std::vector<double> th(nb), rel(nb);
  auto read_status = [&]() {
    for (int j = 0; j < nb; ++j) {
      th[j] = hstat[j];
      rel[j] = std::sqrt(std::max(hstat[nb + j], 0.0)) / std::max(std::fabs(th[j]), 1e-300);
    }
  };
  read_status();
  c.trace(0, 0, th.data(), rel.data(), nev);
  for (int j = 0; j < nev; ++j) lp_prev += th[j];
  bool conv = true;
  for (int j = 0; j < nev; ++j) conv = conv && rel[j] < c.o.tol;
  int it = 0;
  bool hasP = false;
  bool refresh_hs = false;
  int since_refresh = 0;
  double* hC = hstat + 2 * nb + 8;   // host copy of C (k x nb)
  double* hG = hC + (size_t)kmax * nb;  // host copy of G (k x k)
  *reason = 0;
  while (!conv && it < maxiter) {
    if (stop) {
      const int r = stop(it, th.data(), rel.data(), nb);
      if (r) { *reason = r; break; }
    }
    ++it;
    if (refresh_hs && hasP) {
      // HX and HP are carried by the recurrences HX' = HX C1 + HP', HP' = HW C2 + HP C3; with
      // large coefficients (a nearly dependent basis) their rounding drifts away from H X, H P
      // and the next projected problem would be inconsistent: recompute both
      EIG_TRY(c.spmm(X, HX, nb, vt, nb));
      EIG_TRY(c.spmm(P, HP, nb, vt, nb));
      refresh_hs = false;
      since_refresh = 0;
    }
    EIG_TRY(c.spmm(W, HW, nb, vt, nb));
    // Gram blocks: S = [X W P], HS = [HX HW HP]
    BlockList bl;
    int pa[12], pb[12], np = 0;
    PairMap mG, mA;
    for (auto& r : mG.idx) for (int& v : r) v = -1;
    for (auto& r : mA.idx) for (int& v : r) v = -1;
    const int ns = hasP ? 3 : 2;
    if (hasP) {
      bl.n = 6;
      bl.p[0] = X; bl.p[1] = W; bl.p[2] = P; bl.p[3] = HX; bl.p[4] = HW; bl.p[5] = HP;
    } else {
      bl.n = 4;
      bl.p[0] = X; bl.p[1] = W; bl.p[2] = HX; bl.p[3] = HW;
    }
    for (int a = 0; a < ns; ++a)
      for (int b = a; b < ns; ++b) { pa[np] = a; pb[np] = b; mG.idx[a][b] = np; ++np; }
    for (int a = 0; a < ns; ++a)
      for (int b = a; b < ns; ++b) { pa[np] = a; pb[np] = ns + b; mA.idx[a][b] = np; ++np; }
    EIG_TRY(gram_multi(bl, pa, pb, np, nb, n, vt, Gp, gpart, c.st));
    int k = ns * nb;
    k_assemble<<<4, 256, 0, c.st>>>(Gp, mG, ns, nb, G);
    EIG_LAUNCH_CHECK("k_assemble");
    k_assemble<<<4, 256, 0, c.st>>>(Gp, mA, ns, nb, A);
    EIG_LAUNCH_CHECK("k_assemble");
    EIG_TRY(small_rr(A, G, k, nb, piv_tol, theta, C, nullptr, rrwork, info, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat + 2 * nb, info, 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    if (*reinterpret_cast<int*>(hstat + 2 * nb) != SMALL_OK) {
      // the basis lost rank (converged columns' W, or W close to P): Rayleigh-Ritz on the
      // columns a pivoted Cholesky keeps (the others get zero coefficients)
      EIG_TRY(small_rr(A, G, k, nb, piv_tol, theta, C, nullptr, rrwork, info, c.st, 1));
      EIG_CUDA_TRY(cudaMemcpyAsync(hstat + 2 * nb, info, 8, cudaMemcpyDeviceToHost, c.st));
      EIG_TRY(c.sync());
    }
    if (*reinterpret_cast<int*>(hstat + 2 * nb) != SMALL_OK && hasP) {
      // drop P (restart the search direction) and retry on [X W]
      k = 2 * nb;
      PairMap g2, a2;
      for (auto& r : g2.idx) for (int& v : r) v = -1;
      for (auto& r : a2.idx) for (int& v : r) v = -1;
      for (int a = 0; a < 2; ++a)
        for (int b = a; b < 2; ++b) { g2.idx[a][b] = mG.idx[a][b]; a2.idx[a][b] = mA.idx[a][b]; }
      k_assemble<<<4, 256, 0, c.st>>>(Gp, g2, 2, nb, G);
      EIG_LAUNCH_CHECK("k_assemble");
      k_assemble<<<4, 256, 0, c.st>>>(Gp, a2, 2, nb, A);
      EIG_LAUNCH_CHECK("k_assemble");
      EIG_TRY(small_rr(A, G, k, nb, piv_tol, theta, C, nullptr, rrwork, info, c.st));
      EIG_CUDA_TRY(cudaMemcpyAsync(hstat + 2 * nb, info, 8, cudaMemcpyDeviceToHost, c.st));
      EIG_TRY(c.sync());
    }
    if (*reinterpret_cast<int*>(hstat + 2 * nb) != SMALL_OK) {
      *reason = 4;  // the basis lost rank: keep the last Ritz pairs
      --it;
      break;
    }
    {
      // coefficients on unit-norm basis columns: |C_ij| sqrt(G_ii); large ones amplify the
      // rounding of the carried products
      EIG_CUDA_TRY(cudaMemcpyAsync(hC, C, (size_t)k * nb * 8, cudaMemcpyDeviceToHost, c.st));
      EIG_CUDA_TRY(cudaMemcpyAsync(hG, G, (size_t)k * k * 8, cudaMemcpyDeviceToHost, c.st));
      EIG_TRY(c.sync());
      double cmax = 0.0;
      for (int i = 0; i < k; ++i) {
        const double sg = std::sqrt(std::max(hG[(size_t)i * k + i], 0.0));
        for (int j = 0; j < nb; ++j) cmax = std::max(cmax, std::fabs(hC[(size_t)i * nb + j]) * sg);
      }
      if (cmax > 1e3 || ++since_refresh >= 20) refresh_hs = true;
    }
    int nparts = 0;
    EIG_TRY(lobpcg_update(X, W, P, HX, HW, HP, C, k, nb, theta, diagH, c.o.precond_floor, upd_precond(), n, vt, upart,
                          ugrid, &nparts, c.st));
    EIG_TRY(reduce_partials(upart, nparts, nb, rsq, c.st));
    if (lp_on) EIG_TRY(lp_precondition(c, W, HW, nb, nb, vt, theta, rsq, nullptr, nb, W, nonfin));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat, stat, (2 * nb + 2) * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    hasP = true;
    read_status();
    if (lp_on) {
      // Jacobi replaces the learned K once a step raised the wanted Ritz values' sum or an
      // entry of m r was not finite
      double sum = 0.0;
      for (int j = 0; j < nev; ++j) sum += th[j];
      const int bad = *reinterpret_cast<const int*>(hstat + 2 * nb + 1);
      if (bad > 0 || (it > 1 && sum > lp_prev + 1e-6 * std::max(1.0, std::fabs(lp_prev)))) {
        lp_on = false;
        c.s->precond_fallback |= std::min(it, 0xFFFF);
      }
      lp_prev = sum;
    }
    c.trace(0, it, th.data(), rel.data(), nev);
    conv = true;
    for (int j = 0; j < nev; ++j) conv = conv && rel[j] < c.o.tol;
  }
  *iters = it;
  *converged = conv;
  theta_out->assign(th.begin(), th.end());
  if (X64_out) EIG_TRY(convert(X, vt, X64_out, EIG_F64, n * nb, c.st));
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// batched RMM-DIIS (Alg. 4), FP32 vectors: double-float iterates, small quantities in FP32
// (rmm_mixed.cu); same window, DIIS solve and 2x2 Rayleigh-Ritz as the FP64 step below
// ---------------------------------------------------------------------------------------
// RMM-DIIS stall rule: the worst relative residual of the wanted columns that are still
// active has not halved within kRmmStall iterations (columns caught between near-degenerate
// eigenvectors keep RMM-DIIS from converging, Sec. 3.3); the hybrid then hands over to LOBPCG.
// Applied to the FP32-vector RMM-DIIS of the hybrid when its safety net is on (rmm_fallback);
// without it RMM-DIIS runs to its iteration limit, as Alg. 4 does.
constexpr int kRmmStall = 16;
struct RmmStall {
  double best = INFINITY;
  int since = 0;
  bool update(const std::vector<double>& rel, const std::vector<int>& act, int nev) {
    double worst = 0.0;
    for (int j = 0; j < nev; ++j)
      if (act[j]) worst = std::max(worst, rel[j]);
    if (worst < 0.5 * best) {
      best = worst;
      since = 0;
    } else {
      ++since;
    }
    return since >= kRmmStall;
  }
};

static eig_status run_rmmdiis_mixed(Ctx& c, const double* X0, int maxiter, int* iters, bool* converged,
                                    std::vector<double>* theta_out) {
  Handle* h = c.h;
  const int nev = h->n_ev, mp = next_pow2(nev);
  const int64_t n = h->n;
  const int smax = std::max(1, std::min(c.o.s_max, kRmmSMax));
  if (mp > 32) return EIG_EUNSUPPORTED;
  const size_t slab = (size_t)n * mp;
  // big: x history (double-float), r history (FP32), x~ (double-float), r_raw, w, Hw (FP32),
  // and the FP64 start block and its product
  // learned K^{-1} of the corrections (rmm_precond = 2): one more FP32 block for r~
  const bool lp_req = c.o.rmm_precond == 2;
  if (lp_req && !c.o.lp_params) return EIG_EINVAL;
  bool lp_on = lp_req;
  const size_t big_bytes = smax * slab * 8 + smax * slab * 4 + slab * 8 + 3 * slab * 4 + 2 * slab * 8 + 8 * 256 +
                           (lp_req ? slab * 4 + 256 : 0);
  EIG_TRY(h->big.reserve(big_bytes));
  Carve bc(h->big.p, h->big.bytes);
  float2* xh = bc.take<float2>(smax * slab);
  float* rh = bc.take<float>(smax * slab);
  float2* xt = bc.take<float2>(slab);
  float* rraw = bc.take<float>(slab);
  float* w = bc.take<float>(slab);
  float* hw = bc.take<float>(slab);
  double* xs = bc.take<double>(slab);
  double* hxs = bc.take<double>(slab);
  float* rt = lp_req ? bc.take<float>(slab) : nullptr;
  const int grid = std::max(rmx_grid(n, mp), rmm_grid(n, mp));
  const size_t small_bytes = (size_t)mp * kRmmSMax * kRmmSMax * 8 + mp * kRmmSMax * 8 + mp * 3 * kRmmSMax * 4 +
                             mp * 5 * 8 + mp * 8 * 2 + mp * 4 + 2 * kRmmSMax * mp * 8 + mp * 8 +
                             (size_t)grid * mp * (1 + kRmmSMax) * 8 + mp * (1 + kRmmSMax) * 8 * 3 +
                             colsum_scratch_bytes(mp) + 16 * 256 + mp * 16 + 3 * 256;
  EIG_TRY(h->small.reserve(small_bytes));
  Carve cv(h->small.p, h->small.bytes);
  double* B = cv.take<double>((size_t)mp * kRmmSMax * kRmmSMax);
  double* alpha = cv.take<double>((size_t)mp * kRmmSMax);
  float* coef = cv.take<float>((size_t)mp * 3 * kRmmSMax);
  double* par = cv.take<double>(mp * 5);
  double* sg = cv.take<double>((size_t)kRmmSMax * mp);
  double* theta = cv.take<double>(mp);
  double* xn2 = cv.take<double>(mp);
  int* active = cv.take<int>(mp);
  double* thh = cv.take<double>(kRmmSMax * mp);
  double* part = cv.take<double>((size_t)grid * mp * (1 + kRmmSMax));
  double* sums = cv.take<double>((size_t)mp * (1 + kRmmSMax));
  double* s1 = cv.take<double>((size_t)mp * (1 + kRmmSMax));
  double* s2 = cv.take<double>((size_t)mp * (1 + kRmmSMax));
  void* cpart = cv.take<unsigned char>(colsum_scratch_bytes(mp));
  double* th_t = cv.take<double>(mp);
  double* rsq_t = cv.take<double>(mp);
  int* nonfin = cv.take<int>(2);
  if (!bc.ok() || !cv.ok()) return EIG_EUNSUPPORTED;
  EIG_TRY(h->host.reserve(mp * 2 * 8 + 64));
  double* hstat = h->host.as<double>();
  EIG_CUDA_TRY(cudaMemsetAsync(nonfin, 0, 8, c.st));
  EIG_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)mp * kRmmSMax * kRmmSMax * 8, c.st));
  // x^(0): accurate H x^(0) (double-float SpMM), theta^(0), r^(0) (Alg. 4 lines 2-4)
  EIG_TRY(pad_columns(X0, nev, xs, mp, n, c.st));
  EIG_TRY(col_sumsq(xs, mp, n, EIG_F64, xn2, cpart, c.st));
  EIG_TRY(c.spmm(xs, hxs, mp, EIG_F64, nev));
  {
    const int threads = (256 / mp) * mp;
    const int g2 = rmm_grid(n, mp);
    k_coldot2<<<g2, threads, 0, c.st>>>(xs, hxs, nullptr, mp, n, part);
    EIG_LAUNCH_CHECK("k_coldot2");
    EIG_TRY(reduce_partials(part, g2, mp * 2, sums, c.st));
    std::vector<double> hs(mp * 2);
    EIG_CUDA_TRY(cudaMemcpyAsync(hs.data(), sums, mp * 2 * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    std::vector<double> num(mp);
    for (int j = 0; j < mp; ++j) num[j] = hs[j * 2];
    EIG_CUDA_TRY(cudaMemcpyAsync(s1, num.data(), mp * 8, cudaMemcpyHostToDevice, c.st));
    int np = 0;
    {
      std::vector<double> ones((size_t)kRmmSMax * mp, 1.0);
      EIG_CUDA_TRY(cudaMemcpyAsync(sg, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, c.st));
    }
    EIG_TRY(rmx_start(xs, hxs, s1, xn2, mp, n, 0, xh, rh, thh, theta, part, &np, c.st));
    EIG_TRY(reduce_partials(part, np, mp * 2, sums, c.st));
    Window w0;
    w0.s = 1;
    w0.slot[0] = 0;
    EIG_TRY(rmm_store_gram(B, sums, w0, 0, mp, c.st));
    std::vector<double> hs2(mp * 2);
    EIG_CUDA_TRY(cudaMemcpyAsync(hs2.data(), sums, mp * 2 * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat, theta, mp * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    for (int j = 0; j < mp; ++j) hstat[mp + j] = hs2[j * 2];
  }
  std::vector<double> th(mp), rel(mp);
  std::vector<int> act(mp, 0);
  auto refresh = [&]() {
    bool all = true;
    for (int j = 0; j < mp; ++j) {
      th[j] = hstat[j];
      rel[j] = std::sqrt(std::max(hstat[mp + j], 0.0)) / std::max(std::fabs(th[j]), 1e-300);
      act[j] = (j < nev && !(rel[j] < c.o.tol)) ? 1 : 0;
      if (act[j]) all = false;
    }
    return all;
  };
  bool done = refresh();
  c.trace(1, 0, th.data(), rel.data(), nev);
  int count = 1, newest = 0, it = 0;
  RmmStall stall;
  while (!done && it < maxiter) {
    ++it;
    EIG_CUDA_TRY(cudaMemcpyAsync(active, act.data(), mp * 4, cudaMemcpyHostToDevice, c.st));
    Window win;
    win.s = std::min(count, smax);
    for (int i = 0; i < win.s; ++i) win.slot[i] = ((newest - (win.s - 1 - i)) % smax + smax) % smax;
    EIG_TRY(rmm_diis(B, win, active, mp, alpha, c.st, c.o.diis_tol > 0.0 ? c.o.diis_tol : 1e-6));
    EIG_TRY(rmx_coef(alpha, thh, sg, win, newest, mp, coef, c.st));
    const double* tref = thh + (size_t)newest * mp;
    int np = 0;
    EIG_TRY(rmx_combine(xh, rh, coef, win, newest, active, mp, n, xt, rraw, c.o.rmm_precond ? nullptr : w, part, &np,
                        c.st));
    EIG_TRY(reduce_partials(part, np, mp * 3, s1, c.st));
    int nact = 0;
    for (int j = 0; j < mp; ++j) nact += act[j];
    if (lp_on) {
      EIG_TRY(rmx_shifted(xt, rraw, s1, tref, active, mp, n, rt, th_t, c.st));
      EIG_TRY(col_sumsq(rt, mp, n, EIG_F32, rsq_t, cpart, c.st));
      EIG_TRY(lp_precondition(c, rt, hw, mp, mp, EIG_F32, th_t, rsq_t, active, nact, w, nonfin));
    } else if (c.o.rmm_precond) {
      EIG_TRY(rmx_precond(xt, rraw, s1, tref, active, h->plan.diag.as<double>(), c.o.precond_floor, mp, n, w, c.st));
    }
    EIG_TRY(c.rmm_product(w, hw, mp, EIG_F32, act, nev));
    EIG_TRY(rmx_dots(xt, w, rraw, hw, tref, mp, n, part, &np, c.st));
    EIG_TRY(reduce_partials(part, np, mp * 5, s2, c.st));
    EIG_TRY(rmx_rr2(s1, s2, tref, active, mp, theta, par, c.st));
    const int slot_new = (count < smax) ? count : (newest + 1) % smax;
    Window wa;
    wa.s = std::min(count + 1, smax);
    for (int i = 0; i < wa.s; ++i) wa.slot[i] = ((slot_new - (wa.s - 1 - i)) % smax + smax) % smax;
    EIG_TRY(rmx_update(xt, w, rraw, hw, par, slot_new, wa, mp, n, xh, rh, thh, sg, part, &np, c.st));
    EIG_TRY(reduce_partials(part, np, mp * (1 + wa.s), sums, c.st));
    EIG_TRY(rmx_store_gram(B, sums, sg, wa, slot_new, mp, c.st));
    std::vector<double> hs((size_t)mp * (1 + wa.s));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs.data(), sums, hs.size() * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat, theta, mp * 8, cudaMemcpyDeviceToHost, c.st));
    if (lp_on) EIG_CUDA_TRY(cudaMemcpyAsync(hstat + 2 * mp, nonfin, 4, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    for (int j = 0; j < mp; ++j) hstat[mp + j] = hs[(size_t)j * (1 + wa.s)];
    ++count;
    newest = slot_new;
    const double prev_sum = lp_on ? [&]() { double t = 0.0; for (int j = 0; j < nev; ++j) t += th[j]; return t; }()
                                  : 0.0;
    done = refresh();
    if (!done && c.o.rmm_fallback && stall.update(rel, act, nev)) {
      c.trace(1, it, th.data(), rel.data(), nev);
      break;
    }
    if (lp_on) {
      // Jacobi replaces the learned K once a step raised the wanted Ritz values' sum or an
      // entry of m r was not finite
      double sum = 0.0;
      for (int j = 0; j < nev; ++j) sum += th[j];
      const int bad = *reinterpret_cast<const int*>(hstat + 2 * mp);
      if (bad > 0 || sum > prev_sum + 1e-6 * std::max(1.0, std::fabs(prev_sum))) {
        lp_on = false;
        c.s->precond_fallback |= std::min(it, 0xFFFF) << 16;
      }
    }
    c.trace(1, it, th.data(), rel.data(), nev);
  }
  *iters = it;
  *converged = done;
  theta_out->assign(th.begin(), th.begin() + nev);
  EIG_TRY(h->Xres.reserve((size_t)n * nev * 8));
  EIG_TRY(rmx_export(xh + (size_t)newest * slab, sg + (size_t)newest * mp, mp, nev, n, h->Xres.as<double>(), c.st));
  EIG_TRY(c.sync());
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// batched RMM-DIIS (Alg. 4)
// ---------------------------------------------------------------------------------------
eig_status run_rmmdiis(Ctx& c, const double* X0, int maxiter, int* iters, bool* converged,
                       std::vector<double>* theta_out) {
  if (c.o.vec_type == EIG_F32) return run_rmmdiis_mixed(c, X0, maxiter, iters, converged, theta_out);
  Handle* h = c.h;
  const int nev = h->n_ev, mp = next_pow2(nev);
  const int64_t n = h->n;
  const eig_dtype vt = c.o.vec_type;
  const size_t sv = dtype_size(vt);
  const int smax = std::max(1, std::min(c.o.s_max, kRmmSMax));
  if (mp > 32) return EIG_EUNSUPPORTED;
  const size_t slab = (size_t)n * mp;
  // big: xh (smax slabs FP64), rh (smax slabs vt), xt, hxt (FP64), rt, hrt (vt)
  const size_t big_bytes = smax * slab * 8 + smax * slab * sv + 2 * slab * 8 + 2 * slab * sv + 4 * 256;
  EIG_TRY(h->big.reserve(big_bytes));
  Carve bc(h->big.p, h->big.bytes);
  double* xh = bc.take<double>(smax * slab);
  unsigned char* rh = bc.take<unsigned char>(smax * slab * sv);
  double* xt = bc.take<double>(slab);
  double* hxt = bc.take<double>(slab);
  unsigned char* rt = bc.take<unsigned char>(slab * sv);
  unsigned char* hrt = bc.take<unsigned char>(slab * sv);
  const int grid = rmm_grid(n, mp);
  const size_t small_bytes = (size_t)mp * kRmmSMax * kRmmSMax * 8 + mp * kRmmSMax * 8 + mp * 6 * 8 + mp * 2 * 8 +
                             mp * 8 * 4 + kRmmSMax * mp * 8 + (size_t)grid * mp * (1 + kRmmSMax) * 8 +
                             mp * (1 + kRmmSMax) * 8 * 2 + colsum_scratch_bytes(mp) + 16 * 256;
  EIG_TRY(h->small.reserve(small_bytes));
  Carve cv(h->small.p, h->small.bytes);
  double* B = cv.take<double>((size_t)mp * kRmmSMax * kRmmSMax);
  double* alpha = cv.take<double>((size_t)mp * kRmmSMax);
  double* dots = cv.take<double>(mp * 6);
  double* g = cv.take<double>(mp * 2);
  double* stat = cv.take<double>(mp * 2);  // theta, rsq
  double* theta = stat;
  double* rsq = stat + mp;
  int* active = cv.take<int>(mp);
  double* thh = cv.take<double>(kRmmSMax * mp);
  double* part = cv.take<double>((size_t)grid * mp * (1 + kRmmSMax));
  double* sums = cv.take<double>((size_t)mp * (1 + kRmmSMax));
  double* sums2 = cv.take<double>((size_t)mp * (1 + kRmmSMax));
  double* xn2 = cv.take<double>(mp);
  void* cpart = cv.take<unsigned char>(colsum_scratch_bytes(mp));
  if (!bc.ok() || !cv.ok()) return EIG_EUNSUPPORTED;
  EIG_TRY(h->host.reserve(mp * 2 * 8 + 64));
  double* hstat = h->host.as<double>();
  EIG_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)mp * kRmmSMax * kRmmSMax * 8, c.st));
  // x^(0): normalise, accurate H x^(0) in FP64 vectors, theta^(0), r^(0) (Alg. 4 lines 2-4)
  EIG_TRY(pad_columns(X0, nev, xt, mp, n, c.st));
  EIG_TRY(col_sumsq(xt, mp, n, EIG_F64, xn2, cpart, c.st));
  EIG_TRY(c.spmm(xt, hxt, mp, EIG_F64, nev));
  {
    const int threads = (256 / mp) * mp;
    k_coldot2<<<grid, threads, 0, c.st>>>(xt, hxt, nullptr, mp, n, part);
    EIG_LAUNCH_CHECK("k_coldot2");
    EIG_TRY(reduce_partials(part, grid, mp * 2, sums, c.st));
    // sums[j*2] = <x, Hx>; rmm_start takes the numerators with stride 2 -> repack on host side
    std::vector<double> hs(mp * 2);
    EIG_CUDA_TRY(cudaMemcpyAsync(hs.data(), sums, mp * 2 * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    std::vector<double> num(mp);
    for (int j = 0; j < mp; ++j) num[j] = hs[j * 2];
    EIG_CUDA_TRY(cudaMemcpyAsync(sums2, num.data(), mp * 8, cudaMemcpyHostToDevice, c.st));
    int np = 0;
    EIG_TRY(rmm_start(xt, hxt, sums2, xn2, mp, n, vt, 0, xh, rh, thh, theta, part, &np, c.st));
    EIG_TRY(reduce_partials(part, np, mp * 2, sums, c.st));
    Window w0;
    w0.s = 1;
    w0.slot[0] = 0;
    // sums[j*2+0] = ||r||^2 (FP64), sums[j*2+1] = <rq, rq>: store_gram expects [mp][1+s]
    EIG_TRY(rmm_store_gram(B, sums, w0, 0, mp, c.st));
    std::vector<double> hs2(mp * 2);
    EIG_CUDA_TRY(cudaMemcpyAsync(hs2.data(), sums, mp * 2 * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat, theta, mp * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    for (int j = 0; j < mp; ++j) hstat[mp + j] = hs2[j * 2];
  }
  std::vector<double> th(mp), rel(mp);
  std::vector<int> act(mp, 0);
  auto refresh = [&]() {
    bool all = true;
    for (int j = 0; j < mp; ++j) {
      th[j] = hstat[j];
      rel[j] = std::sqrt(std::max(hstat[mp + j], 0.0)) / std::max(std::fabs(th[j]), 1e-300);
      act[j] = (j < nev && !(rel[j] < c.o.tol)) ? 1 : 0;
      if (act[j]) all = false;
    }
    return all;
  };
  bool done = refresh();
  c.trace(1, 0, th.data(), rel.data(), nev);
  int count = 1, newest = 0, it = 0;
  while (!done && it < maxiter) {
    ++it;
    EIG_CUDA_TRY(cudaMemcpyAsync(active, act.data(), mp * 4, cudaMemcpyHostToDevice, c.st));
    Window win;
    win.s = std::min(count, smax);
    for (int i = 0; i < win.s; ++i) win.slot[i] = ((newest - (win.s - 1 - i)) % smax + smax) % smax;
    EIG_TRY(rmm_diis(B, win, active, mp, alpha, c.st, c.o.diis_tol > 0.0 ? c.o.diis_tol : (vt == EIG_F32 ? 1e-6 : 1e-13)));
    int np = 0;
    EIG_TRY(rmm_combine(xh, rh, thh, alpha, win, thh + newest * mp, active, mp, n, vt, xt, hxt, rt, part, &np, c.st));
    EIG_TRY(reduce_partials(part, np, mp * 5, sums, c.st));
    if (c.o.rmm_precond)
      EIG_TRY(rmm_precond_resid(xt, hxt, sums, active, h->plan.diag.as<double>(), c.o.precond_floor, mp, n, vt, rt,
                                c.st));
    int nact = 0;
    for (int j = 0; j < mp; ++j) nact += act[j];
    EIG_TRY(c.rmm_product(rt, hrt, mp, vt, act, nev));
    {
      const int threads = (256 / mp) * mp;
      if (vt == EIG_F32) k_rmm_dots4<float><<<grid, threads, 0, c.st>>>(xt, (const float*)rt, (const float*)hrt, mp, n, part);
      else k_rmm_dots4<double><<<grid, threads, 0, c.st>>>(xt, (const double*)rt, (const double*)hrt, mp, n, part);
      EIG_LAUNCH_CHECK("k_rmm_dots4");
      EIG_TRY(reduce_partials(part, grid, mp * 4, sums2, c.st));
    }
    // sums: combine dots [xx, xhx, xr, rr] (stride 4); sums2: [xhr, rhr, xr, rr]
    {
      // pack: k_pack_rmm_dots reads s2 with stride 2 -> build from sums (stride 4) on device
      // (the first two combine dots are <x,x>, <x,Hx>)
      k_pack_rmm_dots<<<1, 32, 0, c.st>>>(sums, sums2, mp, c.o.rmm_precond, dots);
      EIG_LAUNCH_CHECK("k_pack_rmm_dots");
    }
    EIG_TRY(rmm_rr2(dots, active, mp, theta, g, c.st));
    const int slot_new = (count < smax) ? count : (newest + 1) % smax;
    Window wa;
    wa.s = std::min(count + 1, smax);
    for (int i = 0; i < wa.s; ++i) wa.slot[i] = ((slot_new - (wa.s - 1 - i)) % smax + smax) % smax;
    EIG_TRY(rmm_update(xt, hxt, rt, hrt, g, theta, slot_new, wa, mp, n, vt, xh, rh, thh, part, &np, c.st));
    EIG_TRY(reduce_partials(part, np, mp * (1 + wa.s), sums, c.st));
    EIG_TRY(rmm_store_gram(B, sums, wa, slot_new, mp, c.st));
    // status: theta, ||r||^2
    std::vector<double> hs((size_t)mp * (1 + wa.s));
    EIG_CUDA_TRY(cudaMemcpyAsync(hs.data(), sums, hs.size() * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_CUDA_TRY(cudaMemcpyAsync(hstat, theta, mp * 8, cudaMemcpyDeviceToHost, c.st));
    EIG_TRY(c.sync());
    for (int j = 0; j < mp; ++j) hstat[mp + j] = hs[(size_t)j * (1 + wa.s)];
    // inactive columns keep their previous status (their theta/r are re-derived unchanged)
    ++count;
    newest = slot_new;
    done = refresh();
    c.trace(1, it, th.data(), rel.data(), nev);
  }
  *iters = it;
  *converged = done;
  theta_out->assign(th.begin(), th.begin() + nev);
  // result: newest x slot, first nev columns
  EIG_TRY(h->Xres.reserve((size_t)n * nev * 8));
  {
    BlockList in;
    in.n = 1;
    in.p[0] = xh + (size_t)newest * slab;
    std::vector<double> M((size_t)mp * nev, 0.0);
    for (int j = 0; j < nev; ++j) M[(size_t)j * nev + j] = 1.0;
    DevBuf dM;
    EIG_TRY(dM.reserve(M.size() * 8));
    EIG_CUDA_TRY(cudaMemcpyAsync(dM.p, M.data(), M.size() * 8, cudaMemcpyHostToDevice, c.st));
    EIG_TRY(block_apply(in, mp, dM.as<double>(), nev, h->Xres.p, 0.0, n, EIG_F64, c.st));
    EIG_TRY(c.sync());
  }
  return EIG_OK;
}

}  // namespace eig

// =======================================================================================
// C ABI
// =======================================================================================
using namespace eig;

extern "C" {

void eig_default_opts(eig_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->maxiter = 500;
  o->front = EIG_LOBPCG;
  o->switch_tau = 1e-7;
  o->switch_res = 0.0;
  o->switch_after = 0;
  o->s_max = 10;
  o->vec_type = EIG_F32;
  o->precond = 1;
  o->rmm_precond = 0;
  o->precond_floor = 2.0;
  o->cheb_degree = 10;
  o->lambda_ub = 0.0;
  o->lanczos_maxbasis = 600;
  o->lanczos_keep = 0;
  o->rmm_decouple = 0;
  o->X0 = nullptr;
  o->x0_cols = 0;
  o->x0_on_device = 0;
  o->seed = 1;
  o->certify = 1;
  o->timing = 0;
  o->rmm_maxiter = 0;
  o->rmm_fallback = 1;
  o->diis_tol = 0.0;
  o->stream = nullptr;
}

eig_status eig_create(const eig_csr_upper* H, int n_ev, int block, void** handle) {
  return eig_create_ex(H, n_ev, block, EIG_LAYOUT_AUTO, handle);
}

eig_status eig_create_ex(const eig_csr_upper* H, int n_ev, int block, int layout, void** handle) {
  return eig_create_ex2(H, n_ev, block, layout, 0, 0, handle);
}

eig_status eig_create_ex2(const eig_csr_upper* H, int n_ev, int block, int layout, int row_block, int col_block,
                          void** handle) {
  if (!handle || !H) return EIG_EINVAL;
  *handle = nullptr;
  if (n_ev < 1 || block < n_ev || block > 32 || n_ev > H->n) return EIG_EINVAL;
  if (layout < EIG_LAYOUT_AUTO || layout > EIG_LAYOUT_CSR) return EIG_EINVAL;
  Handle* h = new (std::nothrow) Handle();
  if (!h) return EIG_ENOMEM;
  h->n = H->n;
  h->n_ev = n_ev;
  h->nb = next_pow2(block);
  if (h->nb > H->n) h->nb = std::max(n_ev, (int)H->n);
  eig_status s = spmm_plan_build(&h->plan, H, row_block, col_block, layout, 1, nullptr);
  if (s != EIG_OK) {
    cudaDeviceSynchronize();
    delete h;
    return s;
  }
  *handle = h;
  return EIG_OK;
}

eig_status eig_solver_spmm_info(const void* handle, eig_spmm_info* info) {
  if (!handle || !info) return EIG_EINVAL;
  return eig_spmm_plan_info(&static_cast<const Handle*>(handle)->plan, info);
}

void eig_destroy(void* handle) {
  if (!handle) return;
  cudaDeviceSynchronize();
  delete static_cast<Handle*>(handle);
}

static eig_status solve_impl(Ctx& c, eig_method method) {
  Handle* h = c.h;
  const int64_t n = h->n;
  const int nb = h->nb, nev = h->n_ev;
  // initial guess (FP64 device, n x x0c)
  DevBuf x0buf;
  const double* X0 = nullptr;
  int x0c = 0;
  if (c.o.X0 && c.o.x0_cols > 0) {
    x0c = c.o.x0_cols;
    if (c.o.x0_on_device) {
      X0 = c.o.X0;
    } else {
      EIG_TRY(x0buf.reserve((size_t)n * x0c * 8));
      EIG_CUDA_TRY(cudaMemcpyAsync(x0buf.p, c.o.X0, (size_t)n * x0c * 8, cudaMemcpyHostToDevice, c.st));
      X0 = x0buf.as<double>();
    }
  } else {
    x0c = nb;
    EIG_TRY(x0buf.reserve((size_t)n * x0c * 8));
    EIG_TRY(fill_random(x0buf.as<double>(), n * x0c, c.o.seed, c.st));
    X0 = x0buf.as<double>();
  }
  std::vector<double> theta;
  bool conv = false;
  eig_status rc = EIG_OK;
  cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;
  if (c.o.timing) {
    EIG_CUDA_TRY(cudaEventCreate(&t0));
    EIG_CUDA_TRY(cudaEventCreate(&t1));
    EIG_CUDA_TRY(cudaEventCreate(&t2));
    EIG_CUDA_TRY(cudaEventRecord(t0, c.st));
  }
  // certified residuals the hybrid already computed for its fallback decision (reused below)
  std::vector<double> pre_rel;
  bool pre_dup = false, have_pre = false;
  auto front_then_rmm = [&](eig_method front) -> eig_status {
    std::vector<double> prev;
    double best_rel = INFINITY;
    auto stop = [&](int it, const double* th, const double* rel, int count) -> int {
      double mxr = 0.0;
      for (int j = 0; j < nev; ++j) mxr = std::max(mxr, rel[j]);
      // the front has become unstable (Sec. 2.8: LOBPCG near convergence): residuals climbing
      // well above their best -> hand over to RMM-DIIS now
      if (best_rel < 1e-3 && mxr > 4.0 * best_rel) return 5;
      best_rel = std::min(best_rel, mxr);
      double tau = INFINITY;
      if (!prev.empty()) {
        double s2 = 0.0;
        for (int j = 0; j < nev; ++j) {
          const double den = std::fabs(th[j]) < 1e-12 ? 1.0 : th[j];
          const double d = (th[j] - prev[j]) / den;
          s2 += d * d;
        }
        tau = std::sqrt(s2) / nev;
        c.s->last_tau = tau;
      }
      prev.assign(th, th + nev);
      if (c.o.switch_after > 0) return it >= c.o.switch_after ? 3 : 0;
      // gap condition (option switch_gap): every wanted Ritz vector is within angle switch_gap of
      // an eigenvector (Davis-Kahan: sin angle <= ||r_j|| / gap_j, gap_j the distance from theta_j
      // to the block's other Ritz values), so that RMM-DIIS, which converges to the eigenvector
      // nearest its start, starts inside the right one's basin
      if (c.o.switch_gap > 0.0) {
        for (int j = 0; j < nev; ++j) {
          double gap = INFINITY;
          if (j > 0) gap = std::min(gap, th[j] - th[j - 1]);
          if (j + 1 < count) gap = std::min(gap, th[j + 1] - th[j]);
          if (rel[j] * std::fabs(th[j]) > c.o.switch_gap * gap) return 0;
        }
      }
      if (c.o.switch_res > 0.0) {
        double mx = 0.0;
        for (int j = 0; j < nev; ++j) mx = std::max(mx, rel[j]);
        if (mx <= c.o.switch_res) return 2;
      }
      if (c.o.switch_tau > 0.0 && tau <= c.o.switch_tau) return 1;
      return 0;
    };
    int it = 0, reason = 0;
    bool fconv = false;
    EIG_TRY(h->tmp64b.reserve((size_t)n * nb * 8));
    DevBuf Xf;
    EIG_TRY(Xf.reserve((size_t)n * nb * 8));
    DevBuf Xs;
    EIG_TRY(Xs.reserve((size_t)n * nev * 8));
    if (front == EIG_LOBPCG) {
      EIG_TRY(run_lobpcg(c, X0, x0c, c.o.maxiter, stop, &it, &reason, &fconv, Xf.as<double>(), &theta));
      // the n_ev lowest Ritz vectors (first n_ev columns, ascending theta)
      BlockList in;
      in.n = 1;
      in.p[0] = Xf.p;
      std::vector<double> M((size_t)nb * nev, 0.0);
      for (int j = 0; j < nev; ++j) M[(size_t)j * nev + j] = 1.0;
      DevBuf dM;
      EIG_TRY(dM.reserve(M.size() * 8));
      EIG_CUDA_TRY(cudaMemcpyAsync(dM.p, M.data(), M.size() * 8, cudaMemcpyHostToDevice, c.st));
      EIG_TRY(block_apply(in, nb, dM.as<double>(), nev, Xs.p, 0.0, n, EIG_F64, c.st));
      EIG_TRY(c.sync());
    } else if (front == EIG_BLOCK_LANCZOS) {
      EIG_TRY(run_block_lanczos(c, X0, x0c, c.o.maxiter, stop, &it, &reason, &fconv, &theta));
      EIG_CUDA_TRY(cudaMemcpyAsync(Xs.p, h->Xres.p, (size_t)n * nev * 8, cudaMemcpyDeviceToDevice, c.st));
      EIG_TRY(c.sync());
    } else {
      return EIG_EINVAL;
    }
    c.s->iterations_front = it;
    c.s->switch_reason = reason;
    if (c.o.timing) EIG_CUDA_TRY(cudaEventRecord(t1, c.st));
    if (fconv) {
      conv = true;
      EIG_TRY(h->Xres.reserve((size_t)n * nev * 8));
      EIG_CUDA_TRY(cudaMemcpyAsync(h->Xres.p, Xs.p, (size_t)n * nev * 8, cudaMemcpyDeviceToDevice, c.st));
      EIG_TRY(c.sync());
      theta.resize(nev);
      return EIG_OK;
    }
    // the front's own Ritz vectors beyond the n_ev wanted ones (its guard columns) are kept for
    // the safety net's start block
    const bool have_guards = front == EIG_LOBPCG && nb > nev;
    if (!have_guards) Xf.release();
    int rit = 0;
    EIG_TRY(run_rmmdiis(c, Xs.as<double>(), c.o.rmm_maxiter > 0 ? c.o.rmm_maxiter : c.o.maxiter, &rit, &conv,
                        &theta));
    c.s->iterations_rmm = rit;
    bool dup = false;
    if (c.o.rmm_fallback) {
      // RMM-DIIS updates its residuals by recurrence; over many iterations in FP32 that estimate
      // drifts from H x - theta x, so the FP64 residuals decide whether it converged
      theta.resize(nev);
      EIG_TRY(certify(c, h->Xres.as<double>(), theta, &pre_rel, &dup));
      for (double r : pre_rel) conv = conv && r <= c.o.tol;
      pre_dup = dup;
      have_pre = conv && !dup;
    }
    if (c.o.rmm_fallback && (!conv || dup)) {
      // LOBPCG on FP64 vectors (a subspace method: it separates what RMM-DIIS let drift together)
      // from the RMM-DIIS vectors, to the requested tolerance
      const eig_dtype vt_saved = c.o.vec_type;
      const int pre_saved = c.o.precond;
      c.o.vec_type = EIG_F64;
      if (c.o.precond == 2) c.o.precond = 1;   // the safety net runs with the Jacobi K
      int fit = 0, freason = 0;
      bool fc = false;
      DevBuf Xf2, X0f;
      EIG_TRY(Xf2.reserve((size_t)n * nb * 8));
      EIG_TRY(X0f.reserve((size_t)n * nev * 8));
      // start from the RMM-DIIS vectors without the ones that repeat another, followed by the
      // front's guard Ritz vectors n_ev .. n_b - 1 (LOBPCG front; otherwise LOBPCG fills the block
      // up with seeded random columns)
      std::vector<int> keep;
      EIG_TRY(independent_columns(c, h->Xres.as<double>(), nev, nev, 0.5, &keep));
      if (keep.empty()) keep.push_back(0);
      const int kk = (int)keep.size();
      const int ng = have_guards ? nb - nev : 0;
      EIG_TRY(X0f.reserve((size_t)n * (kk + ng) * 8));
      ColIdx ci;
      for (int q = 0; q < 32; ++q) ci.c[q] = q < kk ? keep[q] : 0;
      DevBuf Xk, Xg;
      EIG_TRY(Xk.reserve((size_t)n * kk * 8));
      k_gather_columns<<<num_sms() * 8, 256, 0, c.st>>>(h->Xres.as<double>(), nev, ci, kk, Xk.as<double>(), n);
      EIG_LAUNCH_CHECK("k_gather_columns");
      if (ng > 0) {
        ColIdx cg;
        for (int q = 0; q < 32; ++q) cg.c[q] = q < ng ? nev + q : 0;
        EIG_TRY(Xg.reserve((size_t)n * ng * 8));
        k_gather_columns<<<num_sms() * 8, 256, 0, c.st>>>(Xf.as<double>(), nb, cg, ng, Xg.as<double>(), n);
        EIG_LAUNCH_CHECK("k_gather_columns");
      }
      // X0f = [Xk | Xg] (row-major n x (kk + ng))
      EIG_CUDA_TRY(cudaMemcpy2DAsync(X0f.p, (size_t)(kk + ng) * 8, Xk.p, (size_t)kk * 8, (size_t)kk * 8, n,
                                     cudaMemcpyDeviceToDevice, c.st));
      if (ng > 0)
        EIG_CUDA_TRY(cudaMemcpy2DAsync(X0f.as<double>() + kk, (size_t)(kk + ng) * 8, Xg.p, (size_t)ng * 8,
                                       (size_t)ng * 8, n, cudaMemcpyDeviceToDevice, c.st));
      const eig_status fr = run_lobpcg(c, X0f.as<double>(), kk + ng, c.o.maxiter, StopFn(), &fit, &freason, &fc,
                                       Xf2.as<double>(), &theta);
      c.o.vec_type = vt_saved;
      c.o.precond = pre_saved;
      EIG_TRY(fr);
      c.s->iterations_fallback = fit;
      BlockList in;
      in.n = 1;
      in.p[0] = Xf2.p;
      std::vector<double> M((size_t)nb * nev, 0.0);
      for (int j = 0; j < nev; ++j) M[(size_t)j * nev + j] = 1.0;
      DevBuf dM;
      EIG_TRY(dM.reserve(M.size() * 8));
      EIG_CUDA_TRY(cudaMemcpyAsync(dM.p, M.data(), M.size() * 8, cudaMemcpyHostToDevice, c.st));
      EIG_TRY(block_apply(in, nb, dM.as<double>(), nev, h->Xres.p, 0.0, n, EIG_F64, c.st));
      EIG_TRY(c.sync());
      theta.resize(nev);
      conv = fc;
    }
    return EIG_OK;
  };
  switch (method) {
    case EIG_HYBRID:
      rc = front_then_rmm(c.o.front);
      break;
    case EIG_LOBPCG: {
      int it = 0, reason = 0;
      DevBuf Xf;
      EIG_TRY(Xf.reserve((size_t)n * nb * 8));
      rc = run_lobpcg(c, X0, x0c, c.o.maxiter, StopFn(), &it, &reason, &conv, Xf.as<double>(), &theta);
      c.s->iterations_front = it;
      if (rc == EIG_OK) {
        EIG_TRY(h->Xres.reserve((size_t)n * nev * 8));
        BlockList in;
        in.n = 1;
        in.p[0] = Xf.p;
        std::vector<double> M((size_t)nb * nev, 0.0);
        for (int j = 0; j < nev; ++j) M[(size_t)j * nev + j] = 1.0;
        DevBuf dM;
        EIG_TRY(dM.reserve(M.size() * 8));
        EIG_CUDA_TRY(cudaMemcpyAsync(dM.p, M.data(), M.size() * 8, cudaMemcpyHostToDevice, c.st));
        EIG_TRY(block_apply(in, nb, dM.as<double>(), nev, h->Xres.p, 0.0, n, EIG_F64, c.st));
        EIG_TRY(c.sync());
        theta.resize(nev);
        if (reason == 4 && !conv) rc = EIG_EBREAKDOWN;
      }
      break;
    }
    case EIG_RMMDIIS: {
      if (x0c < nev) return EIG_EINVAL;
      DevBuf Xs;
      EIG_TRY(Xs.reserve((size_t)n * nev * 8));
      EIG_TRY(pad_columns(X0, x0c, Xs.as<double>(), nev, n, c.st));
      int rit = 0;
      rc = run_rmmdiis(c, Xs.as<double>(), c.o.maxiter, &rit, &conv, &theta);
      c.s->iterations_rmm = rit;
      EIG_TRY(c.sync());
      break;
    }
    case EIG_LANCZOS: {
      int it = 0;
      rc = run_lanczos(c, X0, x0c, &it, &conv, &theta);
      c.s->iterations_front = it;
      break;
    }
    case EIG_BLOCK_LANCZOS: {
      int it = 0, reason = 0;
      rc = run_block_lanczos(c, X0, x0c, c.o.maxiter, StopFn(), &it, &reason, &conv, &theta);
      c.s->iterations_front = it;
      break;
    }
    case EIG_CHEBFILTER: {
      int it = 0;
      rc = run_chebfsi(c, X0, x0c, &it, &conv, &theta);
      c.s->iterations_front = it;
      break;
    }
    default:
      return EIG_EINVAL;
  }
  if (rc != EIG_OK) return rc;
  if (c.o.timing) EIG_CUDA_TRY(cudaEventRecord(t2, c.st));
  h->theta.assign(theta.begin(), theta.begin() + nev);
  h->have = true;
  // true FP64 residuals of the returned pairs
  std::vector<double> rel;
  bool dup = false;
  if (have_pre) {
    rel = pre_rel;
    dup = pre_dup;
  } else if (c.o.certify) {
    EIG_TRY(certify(c, h->Xres.as<double>(), h->theta, &rel, &dup));
  } else {
    rel.assign(nev, NAN);
  }
  h->relres = rel;
  double mx = 0.0;
  for (double r : rel) mx = std::max(mx, r);
  c.s->max_relres = mx;
  c.s->converged = conv ? 1 : 0;
  if (c.o.timing) {
    EIG_TRY(c.sync());
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t2);
    c.s->time_ms_total = ms;
    if (method == EIG_HYBRID) {
      cudaEventElapsedTime(&ms, t0, t1);
      c.s->time_ms_front = ms;
      cudaEventElapsedTime(&ms, t1, t2);
      c.s->time_ms_rmm = ms;
    }
    double sum = 0.0;
    for (size_t i = 0; i < c.spmm_ev.size(); ++i) {
      cudaEventElapsedTime(&ms, c.spmm_ev[i].first, c.spmm_ev[i].second);
      sum += ms;
      c.s->spmm_ms_by_shape[c.spmm_shape[i]] += ms;
    }
    c.s->time_ms_spmm = sum;
    c.s->spmm_timed = (int64_t)c.spmm_ev.size();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaEventDestroy(t2);
  }
  if (dup) return EIG_EDUPLICATE;
  return conv ? EIG_OK : EIG_ENOT_CONVERGED;
}

eig_status eig_solve(void* handle, eig_method method, const eig_opts* opts, eig_stats* stats) {
  return solve_handle(handle, method, opts, stats, nullptr);
}

}  // extern "C"

namespace eig {
eig_status solve_handle(void* handle, eig_method method, const eig_opts* opts, eig_stats* stats,
                        ProductBatcher* batch) {
  if (!handle) return EIG_EINVAL;
  eig_opts o;
  if (opts) o = *opts;
  else eig_default_opts(&o);
  if (!(o.tol > 0.0) || o.maxiter < 0 || o.s_max < 1 || o.s_max > kRmmSMax) return EIG_EINVAL;
  if (o.vec_type != EIG_F32 && o.vec_type != EIG_F64) return EIG_EINVAL;
  if (o.X0 && o.x0_cols < 1) return EIG_EINVAL;
  if (o.precond < 0 || o.precond > 2 || o.rmm_precond < 0 || o.rmm_precond > 2) return EIG_EINVAL;
  if ((o.precond == 2 || o.rmm_precond == 2) && !o.lp_params) return EIG_EINVAL;
  eig_stats local;
  std::memset(&local, 0, sizeof(local));
  Ctx c;
  c.h = static_cast<Handle*>(handle);
  c.st = as_stream(o.stream);
  c.o = o;
  c.s = &local;
  c.batch = batch;
  eig_status rc = solve_impl(c, method);
  cudaStreamSynchronize(c.st);
  if (stats) *stats = local;
  return rc;
}
}  // namespace eig

extern "C" {

eig_status eig_ritz(void* handle, double* theta, double* X, double* relres, int on_device) {
  if (!handle) return EIG_EINVAL;
  Handle* h = static_cast<Handle*>(handle);
  if (!h->have) return EIG_EINVAL;
  if (theta) std::memcpy(theta, h->theta.data(), h->n_ev * 8);
  if (relres) std::memcpy(relres, h->relres.data(), h->n_ev * 8);
  if (X) {
    EIG_CUDA_TRY(cudaMemcpy(X, h->Xres.p, (size_t)h->n * h->n_ev * 8,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  }
  return EIG_OK;
}

}  // extern "C"
