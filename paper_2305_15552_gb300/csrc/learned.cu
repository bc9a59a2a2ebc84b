// Learned per-row preconditioner: features, MLP inference (weights in the kernel-parameter
// constant bank), fused loss + backward with deterministic reductions, Adam.
//
// The preconditioner K^{-1} of Eq. (wblock) is left open by the paper (Sec. 2.3: K only has to
// approximate H); this one replaces the Jacobi scaling by a per-entry factor m_ij = MLP(f_ij)
// learned from the solver's own residuals (the feature list and the network are in learned.cuh).
#include <cmath>
#include <vector>

#include "dense.cuh"
#include "learned.cuh"

namespace eig {
namespace {

constexpr int kApplyThreads = 256;

// ---------------------------------------------------------------------------------------
// (|H| 1)_i: sum over the full row of |h_ij|, from the upper triangle.  Each stored entry adds
// to its row and, off the diagonal, to its column's row.  Integer (fixed-point) atomics make
// the sum exact and order-independent; scale = 2^e with every row sum < 2^61 / scale.
// ---------------------------------------------------------------------------------------
template <typename V>
__global__ void k_lp_abs_total(const V* __restrict__ val, int64_t nnz, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    s += fabs((double)ValLoad<V>::get(val, e));
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <typename V>
__global__ void k_lp_abs_accumulate(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                    const V* __restrict__ val, double scale,
                                    unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    unsigned long long own = 0;
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
      const unsigned long long q = __double2ull_rn(fabs((double)ValLoad<V>::get(val, e)) * scale);
      own += q;
      const int64_t j = col[e];
      if (j != i) atomicAdd(acc + j, q);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xffffffffu, own, o);
    if (lane == 0 && own) atomicAdd(acc + i, own);
  }
}

__global__ void k_lp_abs_finish(int64_t n, const unsigned long long* __restrict__ acc, double inv_scale,
                                double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)acc[i] * inv_scale;
}

// ---------------------------------------------------------------------------------------
// Features and the network
// ---------------------------------------------------------------------------------------
template <typename T> struct LpAcc { typedef float type; };
template <> struct LpAcc<double> { typedef double type; };

// f0..f5 of row i / column j; sc = sqrt(n) / ||r_j|| (0 for a zero column).
template <typename A>
__device__ __forceinline__ void lp_feature_row(double d, double th, double ra, A r, A hr, A sc, float f[kLpFeat]) {
  f[0] = (float)d;
  f[1] = (float)th;
  f[2] = (float)(d - th);
  f[3] = (float)ra;
  f[4] = (float)(r * sc);
  f[5] = (float)((hr - (A)d * r) * sc);
}

// J = 1 / floor(f2), the Jacobi scale the network corrects.
__device__ __forceinline__ float lp_jscale(float f2) {
  const float mag = fmaxf(fabsf(f2), kLpJacobiFloor);
  return 1.0f / (f2 < 0.0f ? -mag : mag);
}

// ReLU that keeps a NaN (so that a broken network reaches the Jacobi fallback).
__device__ __forceinline__ float lp_relu(float a) { return a > 0.0f ? a : (a == a ? 0.0f : a); }

// Weights from the kernel-parameter bank (compile-time offsets after unrolling).
struct LpConstW {
  const LpParams& P;
  __device__ __forceinline__ float operator()(int i) const { return P.p[i]; }
};
// Weights from shared memory.
struct LpSmemW {
  const float* s;
  __device__ __forceinline__ float operator()(int i) const { return s[i]; }
};

// Inference: max(a, 0) (one instruction); a parameter vector with a non-finite entry is
// caught on the host before the launch (it makes every output non-finite, as the network
// arithmetic would).
template <class WA>
__device__ __forceinline__ float lp_infer(const WA& w, const float f[kLpFeat]) {
  float u[kLpFeat];
#pragma unroll
  for (int q = 0; q < kLpFeat; ++q) u[q] = (f[q] - w(kLpOffMu + q)) / w(kLpOffSigma + q);
  float h1[kLpHid];
#pragma unroll
  for (int k = 0; k < kLpHid; ++k) {
    float a = w(kLpOffB1 + k);
#pragma unroll
    for (int q = 0; q < kLpFeat; ++q) a = fmaf(w(kLpOffW1 + k * kLpFeat + q), u[q], a);
    h1[k] = fmaxf(a, 0.0f);
  }
  float m = w(kLpOffB3);
#pragma unroll
  for (int k = 0; k < kLpHid; ++k) {
    float a = w(kLpOffB2 + k);
#pragma unroll
    for (int l = 0; l < kLpHid; ++l) a = fmaf(w(kLpOffW2 + k * kLpHid + l), h1[l], a);
    m = fmaf(w(kLpOffW3 + k), fmaxf(a, 0.0f), m);
  }
  return m;
}

// Per-column constants of a block (theta_j, sqrt(n)/||r_j||, active) into shared memory.
template <typename A>
__device__ __forceinline__ void lp_column_consts(const double* theta, const double* rsq, const int* active, int m,
                                                 int64_t n, double* sTh, A* sSc, int* sAct) {
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    sTh[j] = theta[j];
    const double q = rsq[j];
    sSc[j] = q > 0.0 ? (A)sqrt((double)n / q) : (A)0;
    sAct[j] = active ? active[j] : 1;
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
k_lp_apply(const __grid_constant__ LpParams prm, const T* R, const T* HR, int ld, int m, int64_t n,
           const double* __restrict__ diagH, const double* __restrict__ rowabs, const double* __restrict__ theta,
           const double* __restrict__ rsq, float floor_, const int* __restrict__ active, T* W, int* nonfinite,
           int broken) {
  typedef typename LpAcc<T>::type A;
  __shared__ double sTh[32];
  __shared__ A sSc[32];
  __shared__ int sAct[32];
  lp_column_consts<A>(theta, rsq, active, m, n, sTh, sSc, sAct);
  const LpConstW w{prm};
  int bad = 0;
  const int64_t cnt = n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m;
    const int j = (int)(e - i * m);
    const size_t o = (size_t)i * ld + j;
    const A r = (A)R[o], hr = (A)HR[o];
    const double d = diagH[i];
    A out = (A)0;
    if (sAct[j]) {
      float f[kLpFeat];
      lp_feature_row<A>(d, sTh[j], rowabs[i], r, hr, sSc[j], f);
      out = broken ? (A)NAN : (A)(lp_jscale(f[2]) * (1.0f + lp_infer(w, f))) * r;
      if (!isfinite(out)) {
        A den = (A)(d - sTh[j]);
        const A mag = den < (A)0 ? -den : den;
        const A fl = mag > (A)floor_ ? mag : (A)floor_;
        den = den < (A)0 ? -fl : fl;
        out = r / den;
        ++bad;
      }
    }
    W[o] = (T)out;
  }
  if (nonfinite && bad) atomicAdd(nonfinite, bad);
}

template <typename T>
__global__ void __launch_bounds__(kApplyThreads)
k_lp_features(const T* __restrict__ R, const T* __restrict__ HR, int ld, int m, int64_t n,
              const double* __restrict__ diagH, const double* __restrict__ rowabs, const double* __restrict__ theta,
              const double* __restrict__ rsq, float* __restrict__ F, float* __restrict__ rout) {
  typedef typename LpAcc<T>::type A;
  __shared__ double sTh[32];
  __shared__ A sSc[32];
  __shared__ int sAct[32];
  lp_column_consts<A>(theta, rsq, nullptr, m, n, sTh, sSc, sAct);
  const int64_t cnt = n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / m;
    const int j = (int)(e - i * m);
    const size_t o = (size_t)i * ld + j;
    const A r = (A)R[o];
    float f[kLpFeat];
    lp_feature_row<A>(diagH[i], sTh[j], rowabs[i], r, (A)HR[o], sSc[j], f);
#pragma unroll
    for (int q = 0; q < kLpFeat; ++q) F[e * kLpFeat + q] = f[q];
    rout[e] = (float)r;
  }
}

__global__ void __launch_bounds__(kApplyThreads)
k_lp_forward(const __grid_constant__ LpParams prm, const float* __restrict__ F, int64_t count, float* __restrict__ mo,
             int broken) {
  const LpConstW w{prm};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    float f[kLpFeat];
#pragma unroll
    for (int q = 0; q < kLpFeat; ++q) f[q] = F[e * kLpFeat + q];
    mo[e] = broken ? NAN : lp_jscale(f[2]) * (1.0f + lp_infer(w, f));
  }
}

int params_broken(const LpParams& prm) {
  for (int i = 0; i < kLpParams; ++i)
    if (!std::isfinite(prm.p[i])) return 1;
  return 0;
}

int apply_grid(int64_t count) {
  const int64_t want = (count + kApplyThreads - 1) / kApplyThreads;
  return (int)min64(max64(want, 1), (int64_t)num_sms() * 8);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Loss of the correction targets and its gradient.  A CTA takes tiles of kGradThreads entries
// (one per thread): forward, dL/dm, backward to the per-entry layer deltas, all staged in
// shared memory; then each thread sums, over the tile, the products that make up its own
// parameters' gradient.  Tile sums (FP32) are added into FP64 per-thread totals; CTA partials
// are reduced in a fixed order, so the result is deterministic.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kGradThreads = 128;
constexpr int kGradSlots = (kLpTrained + kGradThreads - 1) / kGradThreads;   // 11
constexpr int kGradOut = kLpTrained + 1;                                      // + loss
constexpr int kSU = 8;                                                        // row stride of sU
constexpr size_t kGradSmemFloats =
    kLpParams + 3 + (size_t)kGradThreads * (kSU + 4 * kLpHid + 1) + 4;

__global__ void __launch_bounds__(kGradThreads)
k_lp_grad(const float* __restrict__ params, const float* __restrict__ F, const float* __restrict__ rr,
          const float* __restrict__ zz, const double* __restrict__ colw, int64_t n, int m,
          double* __restrict__ part) {
  extern __shared__ __align__(16) float sm[];
  float* sW = sm;                                        // kLpParams (+3 pad)
  float* sU = sW + kLpParams + 3;                        // [T][8]
  float* sH1 = sU + kGradThreads * kSU;                  // [T][32]
  float* sH2 = sH1 + kGradThreads * kLpHid;
  float* sDa2 = sH2 + kGradThreads * kLpHid;
  float* sDa1 = sDa2 + kGradThreads * kLpHid;
  float* sDm = sDa1 + kGradThreads * kLpHid;             // [T]
  float* sOne = sDm + kGradThreads;                      // [1] = 1
  __shared__ double red[kGradThreads];
  __shared__ double sTot[kGradSlots * kGradThreads];    // this thread's parameter totals
  const int t = threadIdx.x;
  for (int i = t; i < kLpParams; i += kGradThreads) sW[i] = params[i];
  if (t == 0) sOne[0] = 1.0f;
  for (int s = 0; s < kGradSlots; ++s) sTot[s * kGradThreads + t] = 0.0;
  __syncthreads();
  const LpSmemW w{sW};
  double loss = 0.0;
  const int64_t cnt = n * m;
  const int64_t ntiles = (cnt + kGradThreads - 1) / kGradThreads;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t e = tile * kGradThreads + t;
    const bool valid = e < cnt;
    // ---- forward
    float u[kLpFeat];
    const float jsc = valid ? lp_jscale(F[e * kLpFeat + 2]) : 0.0f;
#pragma unroll
    for (int q = 0; q < kLpFeat; ++q) {
      u[q] = valid ? (F[e * kLpFeat + q] - w(kLpOffMu + q)) / w(kLpOffSigma + q) : 0.0f;
      sU[t * kSU + q] = u[q];
    }
    float h1[kLpHid];
    uint32_t m1 = 0, m2 = 0;
#pragma unroll
    for (int k = 0; k < kLpHid; ++k) {
      float a = w(kLpOffB1 + k);
#pragma unroll
      for (int q = 0; q < kLpFeat; ++q) a = fmaf(w(kLpOffW1 + k * kLpFeat + q), u[q], a);
      h1[k] = valid ? lp_relu(a) : 0.0f;
      if (a > 0.0f) m1 |= 1u << k;
      sH1[t * kLpHid + k] = h1[k];
    }
    float mo = w(kLpOffB3);
#pragma unroll 1
    for (int k = 0; k < kLpHid; ++k) {
      float a = w(kLpOffB2 + k);
#pragma unroll
      for (int l = 0; l < kLpHid; ++l) a = fmaf(w(kLpOffW2 + k * kLpHid + l), h1[l], a);
      const float h2 = valid ? lp_relu(a) : 0.0f;
      if (a > 0.0f) m2 |= 1u << k;
      sH2[t * kLpHid + k] = h2;
      mo = fmaf(w(kLpOffW3 + k), h2, mo);
    }
    // ---- loss, dL/dm and dL/do = dL/dm * J (m = J (1 + o))
    float dm = 0.0f;
    if (valid) {
      const int j = (int)(e % m);
      const float r = rr[e];
      const double cw = colw[j];
      const float err = jsc * (1.0f + mo) * r - zz[e];
      dm = (float)(2.0 * cw) * r * err * jsc;
      loss += cw * (double)err * (double)err;
    }
    sDm[t] = dm;
    // ---- backward to the layer deltas
    float da2[kLpHid];
#pragma unroll
    for (int k = 0; k < kLpHid; ++k) {
      da2[k] = (m2 >> k & 1u) ? dm * w(kLpOffW3 + k) : 0.0f;
      sDa2[t * kLpHid + k] = da2[k];
    }
#pragma unroll 1
    for (int l = 0; l < kLpHid; ++l) {
      float g = 0.0f;
#pragma unroll
      for (int k = 0; k < kLpHid; ++k) g = fmaf(w(kLpOffW2 + k * kLpHid + l), da2[k], g);
      sDa1[t * kLpHid + l] = (m1 >> l & 1u) ? g : 0.0f;
    }
    __syncthreads();
    // ---- this thread's parameters: sum over the tile of (delta x activation)
#pragma unroll 1
    for (int s = 0; s < kGradSlots; ++s) {
      const int q = t + s * kGradThreads;
      if (q < kLpTrained) {
        const float* pa;
        const float* pb;
        int sa, sb;
        if (q < kLpOffB1 - kLpFixed) {                       // W1[k][l]
          pa = sDa1 + q / kLpFeat; sa = kLpHid; pb = sU + q % kLpFeat; sb = kSU;
        } else if (q < kLpOffW2 - kLpFixed) {                // b1[k]
          pa = sDa1 + (q - (kLpOffB1 - kLpFixed)); sa = kLpHid; pb = sOne; sb = 0;
        } else if (q < kLpOffB2 - kLpFixed) {                // W2[k][l]
          const int x = q - (kLpOffW2 - kLpFixed);
          pa = sDa2 + x / kLpHid; sa = kLpHid; pb = sH1 + x % kLpHid; sb = kLpHid;
        } else if (q < kLpOffW3 - kLpFixed) {                // b2[k]
          pa = sDa2 + (q - (kLpOffB2 - kLpFixed)); sa = kLpHid; pb = sOne; sb = 0;
        } else if (q < kLpOffB3 - kLpFixed) {                // w3[k]
          pa = sDm; sa = 1; pb = sH2 + (q - (kLpOffW3 - kLpFixed)); sb = kLpHid;
        } else {                                             // b3
          pa = sDm; sa = 1; pb = sOne; sb = 0;
        }
        float acc = 0.0f;
#pragma unroll 8
        for (int x = 0; x < kGradThreads; ++x) acc = fmaf(pa[x * sa], pb[x * sb], acc);
        sTot[s * kGradThreads + t] += (double)acc;
      }
    }
    __syncthreads();
  }
  for (int s = 0; s < kGradSlots; ++s) {
    const int q = t + s * kGradThreads;
    if (q < kLpTrained) part[(size_t)blockIdx.x * kGradOut + q] = sTot[s * kGradThreads + t];
  }
  red[t] = loss;
  __syncthreads();
  for (int o = kGradThreads / 2; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) part[(size_t)blockIdx.x * kGradOut + kLpTrained] = red[0];
}

__global__ void k_lp_adam(float* __restrict__ p, const double* __restrict__ g, float* __restrict__ m1,
                          float* __restrict__ m2, double lr, double b1, double b2, double bc1, double bc2, double eps) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kLpTrained) return;
  const int i = kLpFixed + q;
  const double gq = g[q];
  const double a = b1 * (double)m1[i] + (1.0 - b1) * gq;
  const double v = b2 * (double)m2[i] + (1.0 - b2) * gq * gq;
  m1[i] = (float)a;
  m2[i] = (float)v;
  p[i] = (float)((double)p[i] - lr * (a / bc1) / (sqrt(v / bc2) + eps));
}

int grad_grid() { return num_sms() * 2; }

template <typename V>
eig_status row_abs_sum_t(const SpmmPlan& P, double* out, cudaStream_t st) {
  const int64_t n = P.n;
  const int grid = num_sms() * 4;
  DevBuf part, acc;
  EIG_TRY(part.reserve((size_t)grid * 8 + 8));
  EIG_TRY(acc.reserve((size_t)n * 8));
  k_lp_abs_total<V><<<grid, 256, 0, st>>>((const V*)P.val, P.nnz, part.as<double>());
  EIG_LAUNCH_CHECK("k_lp_abs_total");
  double* total_d = part.as<double>() + grid;
  EIG_TRY(reduce_partials(part.as<double>(), grid, 1, total_d, st));
  double total = 0.0;
  EIG_CUDA_TRY(cudaMemcpyAsync(&total, total_d, 8, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  if (!std::isfinite(total)) return EIG_EINVAL;
  // every full-row sum is <= total: choose 2^e with total * 2^e < 2^61
  int ex = 0;
  std::frexp(total > 0.0 ? total : 1.0, &ex);
  const double scale = std::ldexp(1.0, 61 - ex);
  EIG_CUDA_TRY(cudaMemsetAsync(acc.p, 0, (size_t)n * 8, st));
  const int ag = (int)min64((n * 32 + 255) / 256, (int64_t)num_sms() * 16);
  k_lp_abs_accumulate<V><<<ag, 256, 0, st>>>(n, P.rowptr, P.col, (const V*)P.val, scale,
                                             acc.as<unsigned long long>());
  EIG_LAUNCH_CHECK("k_lp_abs_accumulate");
  k_lp_abs_finish<<<(int)min64((n + 255) / 256, (int64_t)num_sms() * 8), 256, 0, st>>>(
      n, acc.as<unsigned long long>(), 1.0 / scale, out);
  EIG_LAUNCH_CHECK("k_lp_abs_finish");
  EIG_CUDA_TRY(cudaStreamSynchronize(st));   // part / acc are released on return
  return EIG_OK;
}

}  // namespace

eig_status lp_row_abs_sum(const SpmmPlan& P, double* out, cudaStream_t st) {
  if (!P.rowptr || !out || P.n < 1) return EIG_EINVAL;
  switch (P.val_type) {
    case EIG_F32: return row_abs_sum_t<float>(P, out, st);
    case EIG_F64: return row_abs_sum_t<double>(P, out, st);
    case EIG_BF16: return row_abs_sum_t<uint16_t>(P, out, st);
  }
  return EIG_EINVAL;
}

eig_status lp_apply(const LpParams& prm, const void* R, const void* HR, int ld, int m, int64_t n, eig_dtype vt,
                    const double* diagH, const double* rowabs, const double* theta, const double* rsq, double floor_,
                    const int* active, void* W, int* nonfinite, cudaStream_t st) {
  if (m < 1 || m > 32 || ld < m || n < 0) return EIG_EINVAL;
  if (n == 0) return EIG_OK;
  const int grid = apply_grid(n * m);
  const int broken = params_broken(prm);
  if (vt == EIG_F32)
    k_lp_apply<float><<<grid, kApplyThreads, 0, st>>>(prm, (const float*)R, (const float*)HR, ld, m, n, diagH, rowabs,
                                                      theta, rsq, (float)floor_, active, (float*)W, nonfinite, broken);
  else if (vt == EIG_F64)
    k_lp_apply<double><<<grid, kApplyThreads, 0, st>>>(prm, (const double*)R, (const double*)HR, ld, m, n, diagH,
                                                       rowabs, theta, rsq, (float)floor_, active, (double*)W,
                                                       nonfinite, broken);
  else
    return EIG_EINVAL;
  EIG_LAUNCH_CHECK("k_lp_apply");
  return EIG_OK;
}

eig_status lp_features(const void* R, const void* HR, int ld, int m, int64_t n, eig_dtype vt, const double* diagH,
                       const double* rowabs, const double* theta, const double* rsq, float* F, float* r,
                       cudaStream_t st) {
  if (m < 1 || m > 32 || ld < m || n < 0) return EIG_EINVAL;
  if (n == 0) return EIG_OK;
  const int grid = apply_grid(n * m);
  if (vt == EIG_F32)
    k_lp_features<float><<<grid, kApplyThreads, 0, st>>>((const float*)R, (const float*)HR, ld, m, n, diagH, rowabs,
                                                         theta, rsq, F, r);
  else if (vt == EIG_F64)
    k_lp_features<double><<<grid, kApplyThreads, 0, st>>>((const double*)R, (const double*)HR, ld, m, n, diagH,
                                                          rowabs, theta, rsq, F, r);
  else
    return EIG_EINVAL;
  EIG_LAUNCH_CHECK("k_lp_features");
  return EIG_OK;
}

eig_status lp_forward(const LpParams& prm, const float* F, int64_t count, float* m_out, cudaStream_t st) {
  if (count < 0) return EIG_EINVAL;
  if (count == 0) return EIG_OK;
  k_lp_forward<<<apply_grid(count), kApplyThreads, 0, st>>>(prm, F, count, m_out, params_broken(prm));
  EIG_LAUNCH_CHECK("k_lp_forward");
  return EIG_OK;
}

size_t lp_grad_workspace_bytes() { return (size_t)grad_grid() * kGradOut * 8 + 256; }

eig_status lp_grad(const float* params, const float* F, const float* r, const float* z, const double* colw,
                   int64_t n, int m, double* out, void* workspace, cudaStream_t st) {
  if (m < 1 || n < 0 || !params || !out || !workspace) return EIG_EINVAL;
  const int grid = grad_grid();
  const size_t smem = kGradSmemFloats * sizeof(float);
  // set on every call: the attribute belongs to the current device
  EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_lp_grad, (int)smem));
  k_lp_grad<<<grid, kGradThreads, smem, st>>>(params, F, r, z, colw, n, m, (double*)workspace);
  EIG_LAUNCH_CHECK("k_lp_grad");
  return reduce_partials((const double*)workspace, grid, kGradOut, out, st);
}

eig_status lp_adam(float* params, const double* grad, float* m1, float* m2, int t, double lr, double beta1,
                   double beta2, double eps, cudaStream_t st) {
  if (t < 1 || !params || !grad || !m1 || !m2) return EIG_EINVAL;
  const double bc1 = 1.0 - std::pow(beta1, t), bc2 = 1.0 - std::pow(beta2, t);
  k_lp_adam<<<(kLpTrained + 255) / 256, 256, 0, st>>>(params, grad, m1, m2, lr, beta1, beta2, bc1, bc2, eps);
  EIG_LAUNCH_CHECK("k_lp_adam");
  return EIG_OK;
}

}  // namespace eig
