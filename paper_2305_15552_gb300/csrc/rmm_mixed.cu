// Batched RMM-DIIS step for FP32 vectors (Alg. 4, batched as in Sec. 4.3), GB300 arithmetic.
//
// sm_103a runs FP64 at 1/64 of its FP32 rate, so a step written in FP64 is bound by the FP64
// pipe long before HBM.  This path keeps every FP64-sized quantity in double-float storage and
// forms everything else as a small difference, in FP32:
//   * iterates x^(i) are stored as (hi, lo) FP32 pairs (8 bytes, ~2^-44 relative);
//   * x~ = sum_i a_i x^(i) (Eq. xsum) is summed in double-float from exact FP32 products (the DIIS
//     coefficients may cancel strongly, so a plain FP32 sum is not enough);
//   * r_raw = H x~ - theta_ref x~ = sum_i a_i r^(i) + sum_i a_i (theta^(i) - theta_ref) x^(i)
//     (H x^(i) = r^(i) + theta^(i) x^(i), no SpMM), theta_ref the newest Rayleigh quotient;
//   * the 2x2 Rayleigh-Ritz (Eqs. rr, xuwg) is solved for the shifted pencil
//     (A - theta_ref B) g = mu B g, whose entries are all small, and theta = theta_ref + mu;
//   * r = H x - theta x of the new iterate = g1 (r_raw - mu x~) + g2 (H w - theta w);
//   * every dot product takes exact FP32 products summed in double-float per thread, then
//     FP64 across threads and CTAs in a fixed order;
//   * the 2x2 step's orientation (g1 <= 0) flips consecutive iterates; the history stores
//     y^(i) = s_i x^(i) with a tracked sign s_i = +-1 chosen so that stored neighbours are aligned,
//     and the signs are folded into the combine coefficients and the residual Gram, so the
//     arithmetic is that of the unflipped iterates.
#include <type_traits>

#include "common.cuh"
#include "rmm.cuh"

namespace eig {

namespace {

constexpr int kThreads = 256;
constexpr int kCoef = 3 * kRmmSMax;   // per column: a'_i (hi), a'_i (lo), g'_i

// (hi, lo) += a * b: exact product, two-sum into hi, errors into lo.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err + pe;
}

// Renormalised double-float sum of (hi, lo) and a small FP32 term d.
__device__ __forceinline__ float2 df_add(float hi, float lo, float d) {
  const float s = hi + d;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (d - bb);
  const float l = lo + err;
  const float h = s + l;
  return make_float2(h, l - (h - s));
}

// CTA reduction of NQ double-float accumulators per thread into part[blockIdx][j][q] (FP64).
template <int NQ>
__device__ void cta_reduce_df(const float (&hi)[NQ], const float (&lo)[NQ], int nq, int mp, double* red,
                              double* __restrict__ part) {
  const int rpp = blockDim.x / mp;
  for (int q = 0; q < nq; ++q) red[threadIdx.x * NQ + q] = (double)hi[q] + (double)lo[q];
  __syncthreads();
  for (int idx = threadIdx.x; idx < mp * nq; idx += blockDim.x) {
    const int jj = idx / nq, q = idx % nq;
    double s = 0.0;
    for (int r = 0; r < rpp; ++r) s += red[(r * mp + jj) * NQ + q];
    part[((size_t)blockIdx.x * mp + jj) * nq + q] = s;
  }
}

// C consecutive FP32 values (C = 1, 2, 4) and C consecutive double-float pairs, 16-byte moves.
template <int C> struct F32v;
template <> struct F32v<1> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[1]) { v[0] = *p; }
  __device__ __forceinline__ static void st(float* p, const float (&v)[1]) { *p = v[0]; }
};
template <> struct F32v<2> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[2]) {
    const float2 a = *reinterpret_cast<const float2*>(p);
    v[0] = a.x; v[1] = a.y;
  }
  __device__ __forceinline__ static void st(float* p, const float (&v)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
};
template <> struct F32v<4> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  __device__ __forceinline__ static void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
// pairs (hi, lo) of C elements = 2C floats
template <int C> struct DFv {
  __device__ __forceinline__ static void ld(const float2* p, float (&h)[C], float (&l)[C]) {
    float t[2 * C];
    const float* q = reinterpret_cast<const float*>(p);
    if constexpr (C == 1) {
      F32v<2>::ld(q, *reinterpret_cast<float(*)[2]>(t));
    } else {
#pragma unroll
      for (int k = 0; k < 2 * C; k += 4) F32v<4>::ld(q + k, *reinterpret_cast<float(*)[4]>(t + k));
    }
#pragma unroll
    for (int c = 0; c < C; ++c) { h[c] = t[2 * c]; l[c] = t[2 * c + 1]; }
  }
  __device__ __forceinline__ static void st(float2* p, const float (&h)[C], const float (&l)[C]) {
    float t[2 * C];
#pragma unroll
    for (int c = 0; c < C; ++c) { t[2 * c] = h[c]; t[2 * c + 1] = l[c]; }
    float* q = reinterpret_cast<float*>(p);
    if constexpr (C == 1) {
      F32v<2>::st(q, *reinterpret_cast<const float(*)[2]>(t));
    } else {
#pragma unroll
      for (int k = 0; k < 2 * C; k += 4) F32v<4>::st(q + k, *reinterpret_cast<const float(*)[4]>(t + k));
    }
  }
};

// Columns per thread: 4 adjacent columns (16-byte moves) when the block is that wide.
template <int C> __host__ __device__ constexpr int cols_ok(int mp) { return mp % C == 0; }

// CTA reduction for threads that own C adjacent columns: thread t owns columns (t % gpr) C + c,
// gpr = mp / C.  Writes part[(blockIdx.x * mp + j) * stride + q0 + q], fixed order.
template <int NQ, int C>
__device__ void cta_reduce_cols(const float (&hi)[NQ][C], const float (&lo)[NQ][C], int mp, double* red,
                                double* __restrict__ part, int stride, int q0) {
  const int gpr = mp / C;
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int c = 0; c < C; ++c) red[(threadIdx.x * NQ + q) * C + c] = (double)hi[q][c] + (double)lo[q][c];
  __syncthreads();
  const int per = blockDim.x / gpr;
  for (int idx = threadIdx.x; idx < mp * NQ; idx += blockDim.x) {
    const int j = idx / NQ, q = idx % NQ;
    const int gc = j / C, c = j % C;
    double s = 0.0;
    for (int k = 0; k < per; ++k) s += red[((gc + k * gpr) * NQ + q) * C + c];
    part[((size_t)blockIdx.x * mp + j) * stride + q0 + q] = s;
  }
}

__global__ void __launch_bounds__(kThreads)
k_rmx_start(const double* __restrict__ x0, const double* __restrict__ hx0, const double* __restrict__ num,
            const double* __restrict__ xnorm2, int mp, int64_t n, int slot, float2* __restrict__ xh,
            float* __restrict__ rh, double* __restrict__ thh, double* __restrict__ theta_out,
            double* __restrict__ part) {
  __shared__ double red[kThreads * 2];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const size_t slab = (size_t)n * mp;
  const double nn = xnorm2[j];
  const double inv = nn > 0.0 ? rsqrt(nn) : 0.0;
  const double th = nn > 0.0 ? num[j] / nn : 0.0;
  float hi[2] = {0.0f, 0.0f}, lo[2] = {0.0f, 0.0f};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const double xv = x0[e] * inv;
    const float rq = (float)(hx0[e] * inv - th * xv);
    const float h = (float)xv;
    xh[slot * slab + e] = make_float2(h, (float)(xv - (double)h));
    rh[slot * slab + e] = rq;
    df_fma(hi[0], lo[0], rq, rq);
  }
  hi[1] = hi[0];
  lo[1] = lo[0];
  if (blockIdx.x == 0 && rr == 0) {
    thh[slot * mp + j] = th;
    theta_out[j] = th;
  }
  cta_reduce_df<2>(hi, lo, 2, mp, red, part);
}

// x~ = sum_i a'_i y^(i) and r_raw = sum_i a'_i ry^(i) + g'_i y^(i), both summed in double-float
// (exact FP32 products; the DIIS combination may cancel strongly), w = r_raw for active columns
// when w is given, and partials <x~,x~>, <x~,r_raw>, <x~,y^(newest)> ([cta][j][3]).
// coef: [mp][kCoef] = a'_i as (hi, lo) pairs, then g'_i (FP32), window order; a'_i = a_i s_i,
// g'_i = a_i (theta_i - theta_ref) s_i.  Each thread handles C adjacent columns of a row.
template <int C>
__global__ void __launch_bounds__(kThreads, 3)
k_rmx_combine(const float2* __restrict__ xh, const float* __restrict__ rh, const float* __restrict__ coef, Window win,
              int newest, const int* __restrict__ active, int mp, int64_t n, float2* __restrict__ xt,
              float* __restrict__ rraw, float* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[kThreads * 3 * C];
  __shared__ float sc[32 * kCoef];
  for (int i = threadIdx.x; i < mp * kCoef; i += blockDim.x) sc[i] = coef[i];
  __syncthreads();
  const int gpr = mp / C;
  const int j0 = (threadIdx.x % gpr) * C;
  const size_t slab = (size_t)n * mp;
  bool act[C];
#pragma unroll
  for (int c = 0; c < C; ++c) act[c] = active[j0 + c] != 0;
  float hi[3][C], lo[3][C];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int c = 0; c < C; ++c) hi[q][c] = lo[q][c] = 0.0f;
  const int64_t ng = n * gpr;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const size_t e = (size_t)(g / gpr) * mp + j0;
    float xs[C], xe[C], rs[C], re[C];
#pragma unroll
    for (int c = 0; c < C; ++c) xs[c] = xe[c] = rs[c] = re[c] = 0.0f;
#pragma unroll
    for (int i = 0; i < kRmmSMax; ++i) {
      if (i < win.s) {
        const size_t base = (size_t)win.slot[i] * slab + e;
        float yh[C], yl[C], ri[C];
        DFv<C>::ld(xh + base, yh, yl);
        F32v<C>::ld(rh + base, ri);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float* cc = sc + (j0 + c) * kCoef;
          const float ah = cc[i], al = cc[kRmmSMax + i], gm = cc[2 * kRmmSMax + i];
          df_fma(xs[c], xe[c], ah, yh[c]);
          xe[c] = fmaf(ah, yl[c], fmaf(al, yh[c], xe[c]));
          df_fma(rs[c], re[c], ah, ri[c]);
          re[c] = fmaf(al, ri[c], fmaf(gm, yh[c], re[c]));
        }
      }
    }
    float xo[C], xl[C], res[C], wv[C], yn[C], ynl[C];
    DFv<C>::ld(xh + (size_t)newest * slab + e, yn, ynl);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float2 x = df_add(xs[c], xe[c], 0.0f);
      xo[c] = x.x;
      xl[c] = x.y;
      res[c] = rs[c] + re[c];
      wv[c] = act[c] ? res[c] : 0.0f;
      df_fma(hi[0][c], lo[0][c], xo[c], xo[c]);
      df_fma(hi[1][c], lo[1][c], xo[c], res[c]);
      df_fma(hi[2][c], lo[2][c], xo[c], yn[c]);
    }
    DFv<C>::st(xt + e, xo, xl);
    F32v<C>::st(rraw + e, res);
    if (w) F32v<C>::st(w + e, wv);
  }
  cta_reduce_cols<3, C>(hi, lo, mp, red, part, 3, 0);
}

// Preconditioned correction w = K^{-1}(r_raw - mu~ x~), mu~ = <x~,r_raw>/<x~,x~> (so that
// r_raw - mu~ x~ = H x~ - theta~ x~ with theta~ the Rayleigh quotient of x~), Jacobi K with
// |H_ii - theta~| floored.  sums: [mp][3] from the combine.  C adjacent columns per thread.
template <int C>
__global__ void __launch_bounds__(kThreads)
k_rmx_precond(const float2* __restrict__ xt, const float* __restrict__ rraw, const double* __restrict__ sums,
              const double* __restrict__ theta_ref, const int* __restrict__ active, const double* __restrict__ diagH,
              double floor_, int mp, int64_t n, float* __restrict__ w) {
  const int gpr = mp / C;
  const int j0 = (threadIdx.x % gpr) * C;
  float mu[C], th[C];
  bool act[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j = j0 + c;
    const double xx = sums[j * 3 + 0];
    const double m = xx > 0.0 ? sums[j * 3 + 1] / xx : 0.0;
    mu[c] = (float)m;
    th[c] = (float)(theta_ref[j] + m);   // the preconditioner only needs FP32 accuracy
    act[c] = active[j] != 0;
  }
  const float fl = (float)floor_;
  const int64_t ng = n * gpr;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = g / gpr;
    const size_t e = (size_t)r * mp + j0;
    const float d = (float)diagH[r];
    float xh[C], xl[C], rv[C], wv[C];
    DFv<C>::ld(xt + e, xh, xl);
    F32v<C>::ld(rraw + e, rv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float den = d - th[c];
      const float mag = fmaxf(fabsf(den), fl);
      den = den < 0.0f ? -mag : mag;
      wv[c] = act[c] ? (rv[c] - mu[c] * xh[c]) / den : 0.0f;
    }
    F32v<C>::st(w + e, wv);
  }
}

// The shifted residual r~ = r_raw - mu x~ of k_rmx_precond, materialised (FP32, zero on
// inactive columns) for the learned preconditioner, and theta~ = theta_ref + mu.
template <int C>
__global__ void __launch_bounds__(kThreads)
k_rmx_shifted(const float2* __restrict__ xt, const float* __restrict__ rraw, const double* __restrict__ sums,
              const double* __restrict__ theta_ref, const int* __restrict__ active, int mp, int64_t n,
              float* __restrict__ rt, double* __restrict__ theta_out) {
  const int gpr = mp / C;
  const int j0 = (threadIdx.x % gpr) * C;
  float mu[C];
  bool act[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int j = j0 + c;
    const double xx = sums[j * 3 + 0];
    const double m = xx > 0.0 ? sums[j * 3 + 1] / xx : 0.0;
    mu[c] = (float)m;
    act[c] = active[j] != 0;
  }
  if (blockIdx.x == 0 && threadIdx.x < mp) {
    const int j = threadIdx.x;
    const double xx = sums[j * 3 + 0];
    theta_out[j] = theta_ref[j] + (xx > 0.0 ? sums[j * 3 + 1] / xx : 0.0);
  }
  const int64_t ng = n * gpr;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = g / gpr;
    const size_t e = (size_t)r * mp + j0;
    float xh[C], xl[C], rv[C], ov[C];
    DFv<C>::ld(xt + e, xh, xl);
    F32v<C>::ld(rraw + e, rv);
#pragma unroll
    for (int c = 0; c < C; ++c) ov[c] = act[c] ? rv[c] - mu[c] * xh[c] : 0.0f;
    F32v<C>::st(rt + e, ov);
  }
}

// Partials [cta][j][5] of <x~,w>, <w,w>, <w,r_raw>, <x~, Hw - theta_ref w>, <w, Hw - theta_ref w>.
template <int C>
__global__ void __launch_bounds__(kThreads)
k_rmx_dots(const float2* __restrict__ xt, const float* __restrict__ w, const float* __restrict__ rraw,
           const float* __restrict__ hw, const double* __restrict__ theta_ref, int mp, int64_t n,
           double* __restrict__ part) {
  __shared__ double red[kThreads * 5 * C];
  const int gpr = mp / C;
  const int j0 = (threadIdx.x % gpr) * C;
  float tr[C];
#pragma unroll
  for (int c = 0; c < C; ++c) tr[c] = (float)theta_ref[j0 + c];
  float hi[5][C], lo[5][C];
#pragma unroll
  for (int q = 0; q < 5; ++q)
#pragma unroll
    for (int c = 0; c < C; ++c) hi[q][c] = lo[q][c] = 0.0f;
  const int64_t ng = n * gpr;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const size_t e = (size_t)(g / gpr) * mp + j0;
    float xh[C], xl[C], wv[C], rv[C], hv[C];
    DFv<C>::ld(xt + e, xh, xl);
    F32v<C>::ld(w + e, wv);
    F32v<C>::ld(rraw + e, rv);
    F32v<C>::ld(hw + e, hv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float sh = fmaf(-tr[c], wv[c], hv[c]);
      df_fma(hi[0][c], lo[0][c], xh[c], wv[c]);
      df_fma(hi[1][c], lo[1][c], wv[c], wv[c]);
      df_fma(hi[2][c], lo[2][c], wv[c], rv[c]);
      df_fma(hi[3][c], lo[3][c], xh[c], sh);
      df_fma(hi[4][c], lo[4][c], wv[c], sh);
    }
  }
  cta_reduce_cols<5, C>(hi, lo, mp, red, part, 5, 0);
}

// Shifted 2x2 pencil per column: B = [b11 b12; b12 b22], A - theta_ref B = [c11 c12; c12 c22];
// lowest mu, g with g^T B g = 1 and g1 <= 0 (the orientation of the FP64 step), theta = theta_ref
// + mu.  s1: combine sums [mp][2] (<x,x>, <x,r_raw>); s2: dots sums [mp][5].
// out: theta (FP64) and par[mp][5] = (g1, g2, mu, theta, sigma) for the update, sigma = +-1 the
// storage sign of the new iterate (aligned with the newest stored y: sign of g1 <x~, y_n>).
__global__ void k_rmx_rr2(const double* __restrict__ s1, const double* __restrict__ s2,
                          const double* __restrict__ theta_ref, const int* __restrict__ active, int mp,
                          double* __restrict__ theta, double* __restrict__ par) {
  const int j = threadIdx.x;
  if (j >= mp) return;
  const double b11 = s1[j * 3 + 0], c11 = s1[j * 3 + 1], xy = s1[j * 3 + 2];
  const double b12 = s2[j * 5 + 0], b22 = s2[j * 5 + 1];
  const double c12 = 0.5 * (s2[j * 5 + 2] + s2[j * 5 + 3]), c22 = s2[j * 5 + 4];
  const double tr = theta_ref[j];
  const double sx = b11 > 0.0 ? rsqrt(b11) : 0.0;
  double g1, g2, mu;
  if (!active[j] || !(b22 > 1e-28 * b11) || sx == 0.0) {
    mu = b11 > 0.0 ? c11 / b11 : 0.0;
    g1 = sx;
    g2 = 0.0;
  } else {
    const double sr = rsqrt(b22);
    const double A11 = c11 * sx * sx, A12 = c12 * sx * sr, A22 = c22 * sr * sr, B12 = b12 * sx * sr;
    const double qa = 1.0 - B12 * B12;
    const double qb = -(A11 + A22 - 2.0 * A12 * B12);
    const double qc = A11 * A22 - A12 * A12;
    const double D = fmax(qb * qb - 4.0 * qa * qc, 0.0);
    const double q = -0.5 * (qb + copysign(sqrt(D), qb));
    const double r1 = (qa != 0.0) ? q / qa : 1e300, r2 = (q != 0.0) ? qc / q : 1e300;
    mu = fmin(r1, r2);
    const double m11 = A11 - mu, m12 = A12 - mu * B12, m22 = A22 - mu;
    double h1, h2;
    if (fabs(m11) + fabs(m12) >= fabs(m12) + fabs(m22)) { h1 = m12; h2 = -m11; }
    else { h1 = m22; h2 = -m12; }
    if (h1 == 0.0 && h2 == 0.0) { h1 = 1.0; h2 = 0.0; }
    const double nrm = h1 * h1 + 2.0 * B12 * h1 * h2 + h2 * h2;
    const double s = rsqrt(fmax(nrm, 1e-300)) * (h1 > 0.0 ? -1.0 : 1.0);
    g1 = h1 * s * sx;
    g2 = h2 * s * sr;
  }
  theta[j] = tr + mu;
  par[j * 5 + 0] = g1;
  par[j * 5 + 1] = g2;
  par[j * 5 + 2] = mu;
  par[j * 5 + 3] = tr + mu;
  par[j * 5 + 4] = (g1 * xy < 0.0) ? -1.0 : 1.0;
}

// x = g1 x~ + g2 w (double-float), r = g1 (r_raw - mu x~) + g2 (Hw - theta w), stored times sigma
// in slot `slot_new` (sign sigma recorded in sg); partials [cta][j][stride] (q = 0) of ||r||^2.
template <int C>
__global__ void __launch_bounds__(kThreads)
k_rmx_update(const float2* __restrict__ xt, const float* __restrict__ w, const float* __restrict__ rraw,
             const float* __restrict__ hw, const double* __restrict__ par, int slot_new, int mp, int64_t n,
             float2* __restrict__ xh, float* __restrict__ rh, double* __restrict__ thh, double* __restrict__ sg,
             double* __restrict__ part, int stride) {
  __shared__ double red[kThreads * C];
  const int gpr = mp / C;
  const int j0 = (threadIdx.x % gpr) * C;
  const size_t slab = (size_t)n * mp;
  float g1h[C], g1l[C], g2[C], mu[C], th[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const double* pj = par + (j0 + c) * 5;
    const double sig = pj[4];
    const double g1 = sig * pj[0];
    g1h[c] = (float)g1;
    g1l[c] = (float)(g1 - (double)g1h[c]);
    g2[c] = (float)(sig * pj[1]);
    mu[c] = (float)pj[2];
    th[c] = (float)pj[3];
  }
  float hi[1][C], lo[1][C];
#pragma unroll
  for (int c = 0; c < C; ++c) hi[0][c] = lo[0][c] = 0.0f;
  const int64_t ng = n * gpr;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const size_t e = (size_t)(g / gpr) * mp + j0;
    float xh_[C], xl_[C], wv[C], rv[C], hv[C], nh[C], nl[C], res[C];
    DFv<C>::ld(xt + e, xh_, xl_);
    F32v<C>::ld(w + e, wv);
    F32v<C>::ld(rraw + e, rv);
    F32v<C>::ld(hw + e, hv);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      // g1 * x~ exactly enough: hi part by two-product, the rest rounded
      const float p = g1h[c] * xh_[c];
      const float pe = fmaf(g1h[c], xh_[c], -p);
      const float pl = fmaf(g1h[c], xl_[c], fmaf(g1l[c], xh_[c], pe));
      const float2 xn = df_add(p, pl, g2[c] * wv[c]);
      nh[c] = xn.x;
      nl[c] = xn.y;
      res[c] = fmaf(g1h[c], fmaf(-mu[c], xh_[c], rv[c]), g2[c] * fmaf(-th[c], wv[c], hv[c]));
      df_fma(hi[0][c], lo[0][c], res[c], res[c]);
    }
    DFv<C>::st(xh + (size_t)slot_new * slab + e, nh, nl);
    F32v<C>::st(rh + (size_t)slot_new * slab + e, res);
  }
  if (blockIdx.x == 0 && threadIdx.x < gpr) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      thh[slot_new * mp + j0 + c] = par[(j0 + c) * 5 + 3];
      sg[slot_new * mp + j0 + c] = par[(j0 + c) * 5 + 4];
    }
  }
  cta_reduce_cols<1, C>(hi, lo, mp, red, part, stride, 0);
}

// Residual Gram row of the new slot: partials [cta][j][stride], q = 1 + blockIdx.y, of
// <ry_new, ry^(win.slot[blockIdx.y])> (the Gram store applies the storage signs).
template <int C>
__global__ void __launch_bounds__(kThreads)
k_rmx_gram(const float* __restrict__ rh, int slot_new, Window win, int mp, int64_t n, double* __restrict__ part,
           int stride) {
  __shared__ double red[kThreads * C];
  const int gpr = mp / C;
  const int j0 = (threadIdx.x % gpr) * C;
  const size_t slab = (size_t)n * mp;
  const float* rn = rh + (size_t)slot_new * slab;
  const float* ri = rh + (size_t)win.slot[blockIdx.y] * slab;
  float hi[1][C], lo[1][C];
#pragma unroll
  for (int c = 0; c < C; ++c) hi[0][c] = lo[0][c] = 0.0f;
  const int64_t ng = n * gpr;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
    const size_t e = (size_t)(g / gpr) * mp + j0;
    float a[C], b[C];
    F32v<C>::ld(rn + e, a);
    F32v<C>::ld(ri + e, b);
#pragma unroll
    for (int c = 0; c < C; ++c) df_fma(hi[0][c], lo[0][c], a[c], b[c]);
  }
  cta_reduce_cols<1, C>(hi, lo, mp, red, part, stride, 1 + blockIdx.y);
}

// coef[j] = (a'_i = a_i s_i split as FP32 hi and lo, g'_i = a'_i (theta_i - theta_ref)), window order.
__global__ void k_rmx_coef(const double* __restrict__ alpha, const double* __restrict__ thh,
                           const double* __restrict__ sg, Window win, int newest, int mp, float* __restrict__ coef) {
  const int j = threadIdx.x;
  if (j >= mp) return;
  const double tr = thh[newest * mp + j];
  float* c = coef + j * kCoef;
  for (int i = 0; i < kRmmSMax; ++i) {
    double a = 0.0, g = 0.0;
    if (i < win.s) {
      const int sl = win.slot[i];
      a = alpha[j * kRmmSMax + i] * sg[sl * mp + j];
      g = a * (thh[sl * mp + j] - tr);
    }
    const float h = (float)a;
    c[i] = h;
    c[kRmmSMax + i] = (float)(a - (double)h);
    c[2 * kRmmSMax + i] = (float)g;
  }
}

// Gram row of the new residual: B[j][new][i] = B[j][i][new] = s_new s_i <ry_new, ry_i>.
__global__ void k_rmx_store_gram(double* __restrict__ B, const double* __restrict__ sums, const double* __restrict__ sg,
                                 Window win, int slot_new, int mp) {
  const int j = threadIdx.x;
  if (j >= mp) return;
  double* Bj = B + (size_t)j * kRmmSMax * kRmmSMax;
  const double* sj = sums + (size_t)j * (1 + win.s);
  const double sn = sg[slot_new * mp + j];
  for (int i = 0; i < win.s; ++i) {
    const int si = win.slot[i];
    const double v = sj[1 + i] * sn * sg[si * mp + j];
    Bj[slot_new * kRmmSMax + si] = v;
    Bj[si * kRmmSMax + slot_new] = v;
  }
}

// Final iterate as FP64: X[r][j] = hi + lo for j < nev.
__global__ void k_rmx_export(const float2* __restrict__ xh, const double* __restrict__ sgn, int mp, int nev, int64_t n,
                             double* __restrict__ X) {
  const int64_t total = n * nev;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nev;
    const int j = (int)(i % nev);
    const float2 v = xh[r * mp + j];
    X[i] = sgn[j] * ((double)v.x + (double)v.y);
  }
}

}  // namespace

int rmx_grid(int64_t n, int mp) {
  const int C = (mp % 4 == 0) ? 4 : mp;
  const int64_t groups = n * (mp / C);
  int64_t g = (groups + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

namespace {
// Calls f with the columns-per-thread count for mp (4 when mp is a multiple of 4, else mp).
template <typename F> eig_status by_cols(int mp, F&& f) {
  if (mp % 4 == 0) return f(std::integral_constant<int, 4>{});
  if (mp == 2) return f(std::integral_constant<int, 2>{});
  return f(std::integral_constant<int, 1>{});
}
}  // namespace

eig_status rmx_start(const double* x0, const double* hx0, const double* num, const double* xnorm2, int mp, int64_t n,
                     int slot, void* xh, float* rh, double* thh, double* theta_out, double* part, int* nparts,
                     cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  k_rmx_start<<<grid, (kThreads / mp) * mp, 0, st>>>(x0, hx0, num, xnorm2, mp, n, slot, (float2*)xh, rh, thh,
                                                     theta_out, part);
  EIG_LAUNCH_CHECK("k_rmx_start");
  *nparts = grid;
  return EIG_OK;
}

eig_status rmx_combine(const void* xh, const float* rh, const float* coef, Window win, int newest, const int* active,
                       int mp, int64_t n, void* xt, float* rraw, float* w, double* part, int* nparts,
                       cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  *nparts = grid;
  return by_cols(mp, [&](auto tag) {
    constexpr int C = decltype(tag)::value;
    k_rmx_combine<C><<<grid, kThreads, 0, st>>>((const float2*)xh, rh, coef, win, newest, active, mp, n, (float2*)xt,
                                                rraw, w, part);
    EIG_LAUNCH_CHECK("k_rmx_combine");
    return EIG_OK;
  });
}

eig_status rmx_precond(const void* xt, const float* rraw, const double* sums, const double* theta_ref,
                       const int* active, const double* diagH, double floor_, int mp, int64_t n, float* w,
                       cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  return by_cols(mp, [&](auto tag) {
    constexpr int C = decltype(tag)::value;
    k_rmx_precond<C><<<grid, kThreads, 0, st>>>((const float2*)xt, rraw, sums, theta_ref, active, diagH, floor_, mp,
                                                n, w);
    EIG_LAUNCH_CHECK("k_rmx_precond");
    return EIG_OK;
  });
}

eig_status rmx_shifted(const void* xt, const float* rraw, const double* sums, const double* theta_ref,
                       const int* active, int mp, int64_t n, float* rt, double* theta_out, cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  return by_cols(mp, [&](auto tag) {
    constexpr int C = decltype(tag)::value;
    k_rmx_shifted<C><<<grid, kThreads, 0, st>>>((const float2*)xt, rraw, sums, theta_ref, active, mp, n, rt,
                                                theta_out);
    EIG_LAUNCH_CHECK("k_rmx_shifted");
    return EIG_OK;
  });
}

eig_status rmx_dots(const void* xt, const float* w, const float* rraw, const float* hw, const double* theta_ref,
                    int mp, int64_t n, double* part, int* nparts, cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  *nparts = grid;
  return by_cols(mp, [&](auto tag) {
    constexpr int C = decltype(tag)::value;
    k_rmx_dots<C><<<grid, kThreads, 0, st>>>((const float2*)xt, w, rraw, hw, theta_ref, mp, n, part);
    EIG_LAUNCH_CHECK("k_rmx_dots");
    return EIG_OK;
  });
}

eig_status rmx_rr2(const double* s1, const double* s2, const double* theta_ref, const int* active, int mp,
                   double* theta, double* par, cudaStream_t st) {
  k_rmx_rr2<<<1, 32, 0, st>>>(s1, s2, theta_ref, active, mp, theta, par);
  EIG_LAUNCH_CHECK("k_rmx_rr2");
  return EIG_OK;
}

eig_status rmx_update(const void* xt, const float* w, const float* rraw, const float* hw, const double* par,
                      int slot_new, Window win_after, int mp, int64_t n, void* xh, float* rh, double* thh, double* sg,
                      double* part, int* nparts, cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  const int stride = 1 + win_after.s;
  *nparts = grid;
  return by_cols(mp, [&](auto tag) {
    constexpr int C = decltype(tag)::value;
    k_rmx_update<C><<<grid, kThreads, 0, st>>>((const float2*)xt, w, rraw, hw, par, slot_new, mp, n, (float2*)xh, rh,
                                               thh, sg, part, stride);
    EIG_LAUNCH_CHECK("k_rmx_update");
    k_rmx_gram<C><<<dim3(grid, win_after.s), kThreads, 0, st>>>(rh, slot_new, win_after, mp, n, part, stride);
    EIG_LAUNCH_CHECK("k_rmx_gram");
    return EIG_OK;
  });
}

eig_status rmx_coef(const double* alpha, const double* thh, const double* sg, Window win, int newest, int mp,
                    float* coef, cudaStream_t st) {
  k_rmx_coef<<<1, 32, 0, st>>>(alpha, thh, sg, win, newest, mp, coef);
  EIG_LAUNCH_CHECK("k_rmx_coef");
  return EIG_OK;
}

eig_status rmx_store_gram(double* B, const double* sums, const double* sg, Window win_after, int slot_new, int mp,
                          cudaStream_t st) {
  k_rmx_store_gram<<<1, 32, 0, st>>>(B, sums, sg, win_after, slot_new, mp);
  EIG_LAUNCH_CHECK("k_rmx_store_gram");
  return EIG_OK;
}

eig_status rmx_export(const void* xh_slot, const double* sgn, int mp, int nev, int64_t n, double* X, cudaStream_t st) {
  k_rmx_export<<<num_sms() * 8, 256, 0, st>>>((const float2*)xh_slot, sgn, mp, nev, n, X);
  EIG_LAUNCH_CHECK("k_rmx_export");
  return EIG_OK;
}

}  // namespace eig
