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
// when w is given, and partials <x~,x~>, <x~,r_raw>, <x~,y^(newest)>.
// coef: [mp][kCoef] = a'_i as (hi, lo) pairs, then g'_i (FP32), window order; a'_i = a_i s_i,
// g'_i = a_i (theta_i - theta_ref) s_i.
__global__ void __launch_bounds__(kThreads)
k_rmx_combine(const float2* __restrict__ xh, const float* __restrict__ rh, const float* __restrict__ coef, Window win,
              int newest, const int* __restrict__ active, int mp, int64_t n, float2* __restrict__ xt,
              float* __restrict__ rraw, float* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[kThreads * 3];
  __shared__ float sc[32 * kCoef];
  for (int i = threadIdx.x; i < mp * kCoef; i += blockDim.x) sc[i] = coef[i];
  __syncthreads();
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const size_t slab = (size_t)n * mp;
  const float* ah = sc + j * kCoef;
  const float* al = ah + kRmmSMax;
  const float* gm = al + kRmmSMax;
  const bool act = active[j] != 0;
  float hi[3] = {0.0f, 0.0f, 0.0f}, lo[3] = {0.0f, 0.0f, 0.0f};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    float xs = 0.0f, xe = 0.0f, rs = 0.0f, re = 0.0f;
#pragma unroll
    for (int i = 0; i < kRmmSMax; ++i) {
      if (i < win.s) {
        const int sl = win.slot[i];
        const float2 yi = xh[sl * slab + e];
        const float ri = rh[sl * slab + e];
        // x: (ah + al) (hi + lo), hi part exact
        df_fma(xs, xe, ah[i], yi.x);
        xe = fmaf(ah[i], yi.y, fmaf(al[i], yi.x, xe));
        // r_raw: (ah + al) ri + g'_i y_i
        df_fma(rs, re, ah[i], ri);
        re = fmaf(al[i], ri, fmaf(gm[i], yi.x, re));
      }
    }
    const float2 x = df_add(xs, xe, 0.0f);
    const float res = rs + re;
    const float yn = xh[newest * slab + e].x;
    xt[e] = x;
    rraw[e] = res;
    if (w) w[e] = act ? res : 0.0f;
    df_fma(hi[0], lo[0], x.x, x.x);
    df_fma(hi[1], lo[1], x.x, res);
    df_fma(hi[2], lo[2], x.x, yn);
  }
  cta_reduce_df<3>(hi, lo, 3, mp, red, part);
}

// Preconditioned correction w = K^{-1}(r_raw - mu~ x~), mu~ = <x~,r_raw>/<x~,x~> (so that
// r_raw - mu~ x~ = H x~ - theta~ x~ with theta~ the Rayleigh quotient of x~), Jacobi K with
// |H_ii - theta~| floored.  sums: [mp][3] from the combine.
__global__ void k_rmx_precond(const float2* __restrict__ xt, const float* __restrict__ rraw,
                              const double* __restrict__ sums, const double* __restrict__ theta_ref,
                              const int* __restrict__ active, const double* __restrict__ diagH, double floor_,
                              int mp, int64_t n, float* __restrict__ w) {
  const int64_t total = n * mp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % mp);
    if (!active[j]) { w[i] = 0.0f; continue; }
    const double xx = sums[j * 3 + 0];
    const double mu = xx > 0.0 ? sums[j * 3 + 1] / xx : 0.0;
    // the preconditioner only needs |H_ii - theta~| to FP32 accuracy
    float den = (float)diagH[i / mp] - (float)(theta_ref[j] + mu);
    const float mag = fmaxf(fabsf(den), (float)floor_);
    den = den < 0.0f ? -mag : mag;
    w[i] = (rraw[i] - (float)mu * xt[i].x) / den;
  }
}

// Partials of <x~,w>, <w,w>, <w,r_raw>, <x~, Hw - theta_ref w>, <w, Hw - theta_ref w>.
__global__ void __launch_bounds__(kThreads)
k_rmx_dots(const float2* __restrict__ xt, const float* __restrict__ w, const float* __restrict__ rraw,
           const float* __restrict__ hw, const double* __restrict__ theta_ref, int mp, int64_t n,
           double* __restrict__ part) {
  __shared__ double red[kThreads * 5];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const float tr = (float)theta_ref[j];
  float hi[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const float x = xt[e].x, wv = w[e], rv = rraw[e];
    const float sh = fmaf(-tr, wv, hw[e]);
    df_fma(hi[0], lo[0], x, wv);
    df_fma(hi[1], lo[1], wv, wv);
    df_fma(hi[2], lo[2], wv, rv);
    df_fma(hi[3], lo[3], x, sh);
    df_fma(hi[4], lo[4], wv, sh);
  }
  cta_reduce_df<5>(hi, lo, 5, mp, red, part);
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
// in slot `slot_new` (sign sigma recorded in sg); partials of ||r||^2 and <sigma r, ry^(i)> for the
// window after the update (the Gram store applies the signs).
__global__ void __launch_bounds__(kThreads)
k_rmx_update(const float2* __restrict__ xt, const float* __restrict__ w, const float* __restrict__ rraw,
             const float* __restrict__ hw, const double* __restrict__ par, int slot_new, Window win, int mp,
             int64_t n, float2* __restrict__ xh, float* __restrict__ rh, double* __restrict__ thh,
             double* __restrict__ sg, double* __restrict__ part) {
  __shared__ double red[kThreads * (1 + kRmmSMax)];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const size_t slab = (size_t)n * mp;
  const double sig = par[j * 5 + 4];
  const double g1 = sig * par[j * 5 + 0], g2d = sig * par[j * 5 + 1];
  const float g1h = (float)g1, g1l = (float)(g1 - (double)g1h), g2 = (float)g2d;
  const float mu = (float)par[j * 5 + 2], th = (float)par[j * 5 + 3];
  float hi[1 + kRmmSMax], lo[1 + kRmmSMax];
#pragma unroll
  for (int q = 0; q <= kRmmSMax; ++q) hi[q] = lo[q] = 0.0f;
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const float2 x = xt[e];
    const float wv = w[e], rv = rraw[e], hv = hw[e];
    // g1 * x~ exactly enough: hi part by two-product, the rest rounded
    const float p = g1h * x.x;
    const float pe = fmaf(g1h, x.x, -p);
    const float pl = fmaf(g1h, x.y, fmaf(g1l, x.x, pe));
    const float2 xn = df_add(p, pl, g2 * wv);
    const float res = fmaf(g1h, fmaf(-mu, x.x, rv), g2 * fmaf(-th, wv, hv));
    xh[slot_new * slab + e] = xn;
    rh[slot_new * slab + e] = res;
    df_fma(hi[0], lo[0], res, res);
#pragma unroll
    for (int i = 0; i < kRmmSMax; ++i) {
      if (i < win.s) {
        const int sl = win.slot[i];
        const float o = (sl == slot_new) ? res : rh[sl * slab + e];
        df_fma(hi[1 + i], lo[1 + i], res, o);
      }
    }
  }
  if (blockIdx.x == 0 && rr == 0) {
    thh[slot_new * mp + j] = par[j * 5 + 3];
    sg[slot_new * mp + j] = sig;
  }
  cta_reduce_df<1 + kRmmSMax>(hi, lo, 1 + win.s, mp, red, part);
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
  const int rpp = kThreads / mp;
  int64_t g = (n + rpp - 1) / rpp;
  const int64_t cap = (int64_t)num_sms() * 6;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

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
  k_rmx_combine<<<grid, (kThreads / mp) * mp, 0, st>>>((const float2*)xh, rh, coef, win, newest, active, mp, n,
                                                       (float2*)xt, rraw, w, part);
  EIG_LAUNCH_CHECK("k_rmx_combine");
  *nparts = grid;
  return EIG_OK;
}

eig_status rmx_precond(const void* xt, const float* rraw, const double* sums, const double* theta_ref,
                       const int* active, const double* diagH, double floor_, int mp, int64_t n, float* w,
                       cudaStream_t st) {
  k_rmx_precond<<<num_sms() * 8, 256, 0, st>>>((const float2*)xt, rraw, sums, theta_ref, active, diagH, floor_, mp,
                                               n, w);
  EIG_LAUNCH_CHECK("k_rmx_precond");
  return EIG_OK;
}

eig_status rmx_dots(const void* xt, const float* w, const float* rraw, const float* hw, const double* theta_ref,
                    int mp, int64_t n, double* part, int* nparts, cudaStream_t st) {
  const int grid = rmx_grid(n, mp);
  k_rmx_dots<<<grid, (kThreads / mp) * mp, 0, st>>>((const float2*)xt, w, rraw, hw, theta_ref, mp, n, part);
  EIG_LAUNCH_CHECK("k_rmx_dots");
  *nparts = grid;
  return EIG_OK;
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
  k_rmx_update<<<grid, (kThreads / mp) * mp, 0, st>>>((const float2*)xt, w, rraw, hw, par, slot_new, win_after, mp,
                                                      n, (float2*)xh, rh, thh, sg, part);
  EIG_LAUNCH_CHECK("k_rmx_update");
  *nparts = grid;
  return EIG_OK;
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
