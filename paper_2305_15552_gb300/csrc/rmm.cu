// Batched RMM-DIIS (Alg. 4, batched as in Sec. 4.3): all n_ev refinements advance in
// lock-step so that their products with H form one SpMM on the block of r~ vectors.
//
// Precision layout: iterates x^(i) in FP64, residual history r^(i) in the SpMM vector type
// (FP32 in the mixed-precision path: residuals are small, so FP32 keeps their relative
// accuracy), the SpMM operand r~ in the vector type and H r~ accumulated into FP64 iterates.
// H x~ is never formed by an SpMM: H x^(i) = r^(i) + theta^(i) x^(i), so
// H x~ = sum_i alpha_i (r^(i) + theta^(i) x^(i)) by linearity, and H x = g1 H x~ + g2 H r~.
#include "common.cuh"
#include "rmm.cuh"

namespace eig {

constexpr int kRmmThreads = 256;

int rmm_grid(int64_t n, int mp) {
  const int rpp = kRmmThreads / mp;
  int64_t g = (n + rpp - 1) / rpp;
  const int64_t cap = (int64_t)num_sms() * 6;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// CTA-level column reduction of NQ values per thread: red is [kRmmThreads][NQ];
// writes part[blockIdx.x][j][q].
template <int NQ>
__device__ void cta_colreduce(double (&v)[NQ], int mp, double* red, double* part) {
  const int j = threadIdx.x % mp, rpp = blockDim.x / mp;
#pragma unroll
  for (int q = 0; q < NQ; ++q) red[threadIdx.x * NQ + q] = v[q];
  __syncthreads();
  for (int idx = threadIdx.x; idx < mp * NQ; idx += blockDim.x) {
    const int jj = idx / NQ, q = idx % NQ;
    double s = 0.0;
    for (int r = 0; r < rpp; ++r) s += red[(r * mp + jj) * NQ + q];
    part[((size_t)blockIdx.x * mp + jj) * NQ + q] = s;
  }
  (void)j;
}

template <typename T>
__global__ void __launch_bounds__(kRmmThreads)
k_rmm_combine(const double* __restrict__ xh, const T* __restrict__ rh, const double* __restrict__ thh,
              const double* __restrict__ alpha, Window win, const double* __restrict__ theta_ref,
              const int* __restrict__ active, int mp, int64_t n, double* __restrict__ xt, double* __restrict__ hxt,
              T* __restrict__ rt, double* __restrict__ part) {
  __shared__ double red[kRmmThreads * 5];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const size_t slab = (size_t)n * mp;
  double a[kRmmSMax], th[kRmmSMax];
  for (int i = 0; i < win.s; ++i) {
    a[i] = alpha[j * kRmmSMax + i];
    th[i] = thh[win.slot[i] * mp + j];
  }
  const double tref = theta_ref[j];
  const bool act = active[j] != 0;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    double x = 0.0, hx = 0.0;
    for (int i = 0; i < win.s; ++i) {
      if (a[i] == 0.0) continue;
      const double xv = xh[win.slot[i] * slab + e];
      const double rv = (double)rh[win.slot[i] * slab + e];
      x = fma(a[i], xv, x);
      hx = fma(a[i], fma(th[i], xv, rv), hx);
    }
    xt[e] = x;
    hxt[e] = hx;
    const T rtv = act ? (T)(hx - tref * x) : T(0);
    rt[e] = rtv;
    const double rd = (double)rtv;
    v[0] = fma(x, x, v[0]);
    v[1] = fma(x, hx, v[1]);
    v[2] = fma(x, rd, v[2]);
    v[3] = fma(rd, rd, v[3]);
    v[4] = fma(rd, hx, v[4]);
  }
  cta_colreduce<5>(v, mp, red, part);
}

template <typename T>
__global__ void __launch_bounds__(kRmmThreads)
k_rmm_dots2(const double* __restrict__ xt, const T* __restrict__ rt, const T* __restrict__ hrt, int mp, int64_t n,
            double* __restrict__ part) {
  __shared__ double red[kRmmThreads * 2];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  double v[2] = {0.0, 0.0};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const double h = (double)hrt[e];
    v[0] = fma(xt[e], h, v[0]);
    v[1] = fma((double)rt[e], h, v[1]);
  }
  cta_colreduce<2>(v, mp, red, part);
}

// Preconditioned correction of RMM-DIIS: r~ = K^{-1}(H x~ - theta~ x~), theta~ = <x~,Hx~>/<x~,x~>
// taken from the combine sums (stride 5); Jacobi K with |H_ii - theta~| floored.
template <typename T>
__global__ void k_rmm_precond_resid(const double* __restrict__ xt, const double* __restrict__ hxt,
                                    const double* __restrict__ sums, const int* __restrict__ active,
                                    const double* __restrict__ diagH, double floor, int mp, int64_t n,
                                    T* __restrict__ rt) {
  const int64_t total = n * mp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % mp);
    if (!active[j]) { rt[i] = T(0); continue; }
    const double xx = sums[j * 5 + 0];
    const double th = xx > 0.0 ? sums[j * 5 + 1] / xx : 0.0;
    double den = diagH[i / mp] - th;
    const double mag = fmax(fabs(den), floor);
    den = den < 0.0 ? -mag : mag;
    rt[i] = (T)((hxt[i] - th * xt[i]) / den);
  }
}

eig_status rmm_precond_resid(const double* xt, const double* hxt, const double* sums, const int* active,
                             const double* diagH, double floor, int mp, int64_t n, eig_dtype vt, void* rt,
                             cudaStream_t st) {
  const int grid = num_sms() * 8;
  if (vt == EIG_F32)
    k_rmm_precond_resid<float><<<grid, 256, 0, st>>>(xt, hxt, sums, active, diagH, floor, mp, n, (float*)rt);
  else
    k_rmm_precond_resid<double><<<grid, 256, 0, st>>>(xt, hxt, sums, active, diagH, floor, mp, n, (double*)rt);
  EIG_LAUNCH_CHECK("k_rmm_precond_resid");
  return EIG_OK;
}

__global__ void k_rmm_rr2(const double* __restrict__ dots, const int* __restrict__ active, int mp,
                          double* __restrict__ theta, double* __restrict__ g) {
  const int j = threadIdx.x;
  if (j >= mp) return;
  const double* d = dots + j * 6;
  const double b11 = d[0], a11 = d[1], b12 = d[2], b22 = d[3], a12 = d[4], a22 = d[5];
  const double sx = b11 > 0.0 ? rsqrt(b11) : 0.0;
  if (!active[j] || !(b22 > 1e-28 * b11) || sx == 0.0) {
    theta[j] = b11 > 0.0 ? a11 / b11 : 0.0;
    g[2 * j] = sx;
    g[2 * j + 1] = 0.0;
    return;
  }
  const double sr = rsqrt(b22);
  // unit-diagonal scaling of the pencil
  const double A11 = a11 * sx * sx, A12 = a12 * sx * sr, A22 = a22 * sr * sr, B12 = b12 * sx * sr;
  const double qa = 1.0 - B12 * B12;
  const double qb = -(A11 + A22 - 2.0 * A12 * B12);
  const double qc = A11 * A22 - A12 * A12;
  const double D = fmax(qb * qb - 4.0 * qa * qc, 0.0);
  const double q = -0.5 * (qb + copysign(sqrt(D), qb));
  double r1 = (qa != 0.0) ? q / qa : 1e300, r2 = (q != 0.0) ? qc / q : 1e300;
  const double th = fmin(r1, r2);
  // null vector of (A - th B)
  const double m11 = A11 - th, m12 = A12 - th * B12, m22 = A22 - th;
  double g1, g2;
  if (fabs(m11) + fabs(m12) >= fabs(m12) + fabs(m22)) { g1 = m12; g2 = -m11; }
  else { g1 = m22; g2 = -m12; }
  if (g1 == 0.0 && g2 == 0.0) { g1 = 1.0; g2 = 0.0; }
  // g^T B g = 1, and g1 <= 0: consecutive iterates alternate in sign (the DIIS constraint of
  // Eq. alphasum is not sign invariant; this is the orientation LAPACK's generalized solver gives)
  const double nrm = g1 * g1 + 2.0 * B12 * g1 * g2 + g2 * g2;
  const double s = rsqrt(fmax(nrm, 1e-300)) * (g1 > 0.0 ? -1.0 : 1.0);
  theta[j] = th;
  g[2 * j] = g1 * s * sx;
  g[2 * j + 1] = g2 * s * sr;
}

template <typename T>
__global__ void __launch_bounds__(kRmmThreads)
k_rmm_update(const double* __restrict__ xt, const double* __restrict__ hxt, const T* __restrict__ rt,
             const T* __restrict__ hrt, const double* __restrict__ g, const double* __restrict__ theta, int slot_new,
             Window win, int mp, int64_t n, double* __restrict__ xh, T* __restrict__ rh, double* __restrict__ thh,
             double* __restrict__ part) {
  extern __shared__ double red[];  // kRmmThreads * (1 + s)
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const size_t slab = (size_t)n * mp;
  const double g1 = g[2 * j], g2 = g[2 * j + 1], th = theta[j];
  double v[1 + kRmmSMax];
  for (int q = 0; q <= win.s; ++q) v[q] = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const double x = fma(g1, xt[e], g2 * (double)rt[e]);
    const double hx = fma(g1, hxt[e], g2 * (double)hrt[e]);
    const double res = hx - th * x;
    const T rq = (T)res;
    xh[slot_new * slab + e] = x;
    rh[slot_new * slab + e] = rq;
    v[0] = fma(res, res, v[0]);
    const double rd = (double)rq;
    for (int i = 0; i < win.s; ++i) {
      const double o = (win.slot[i] == slot_new) ? rd : (double)rh[win.slot[i] * slab + e];
      v[1 + i] = fma(rd, o, v[1 + i]);
    }
  }
  if (blockIdx.x == 0 && rr == 0) thh[slot_new * mp + j] = th;
  const int NQ = 1 + win.s;
  for (int q = 0; q < NQ; ++q) red[threadIdx.x * NQ + q] = v[q];
  __syncthreads();
  for (int idx = threadIdx.x; idx < mp * NQ; idx += blockDim.x) {
    const int jj = idx / NQ, q = idx % NQ;
    double s = 0.0;
    for (int r2 = 0; r2 < rpp; ++r2) s += red[(r2 * mp + jj) * NQ + q];
    part[((size_t)blockIdx.x * mp + jj) * NQ + q] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRmmThreads)
k_rmm_start(double* __restrict__ x, const double* __restrict__ hx, const double* __restrict__ num,
            const double* __restrict__ xnorm2, int mp, int64_t n, int slot, double* __restrict__ xh,
            T* __restrict__ rh, double* __restrict__ thh, double* __restrict__ theta_out, double* __restrict__ part) {
  __shared__ double red[kRmmThreads * 2];
  const int j = threadIdx.x % mp, rr = threadIdx.x / mp, rpp = blockDim.x / mp;
  const size_t slab = (size_t)n * mp;
  const double nn = xnorm2[j];
  const double inv = nn > 0.0 ? rsqrt(nn) : 0.0;
  const double th = nn > 0.0 ? num[j] / nn : 0.0;
  double v[2] = {0.0, 0.0};
  for (int64_t r = blockIdx.x * (int64_t)rpp + rr; r < n; r += (int64_t)gridDim.x * rpp) {
    const size_t e = (size_t)r * mp + j;
    const double xv = x[e] * inv;
    const double res = hx[e] * inv - th * xv;
    const T rq = (T)res;
    xh[slot * slab + e] = xv;
    rh[slot * slab + e] = rq;
    v[0] = fma(res, res, v[0]);
    v[1] = fma((double)rq, (double)rq, v[1]);
  }
  if (blockIdx.x == 0 && rr == 0) {
    thh[slot * mp + j] = th;
    theta_out[j] = th;
  }
  cta_colreduce<2>(v, mp, red, part);
}

// One warp per column j (CTA j): lane i owns row i of the (s-1)x(s-1) system, kept in shared
// memory; each entry is computed with the same operations in the same order as a sequential
// Cholesky would, so the result does not depend on the parallel layout.
__global__ void __launch_bounds__(32) k_rmm_diis(const double* __restrict__ B, Window win,
                                                 const int* __restrict__ active, int mp, double tol,
                                                 double* __restrict__ alpha) {
  constexpr int M = kRmmSMax - 1;
  __shared__ double F[M][M + 1];
  __shared__ double rhs[M], y[M];
  __shared__ int fail;
  const int j = blockIdx.x, lane = threadIdx.x;
  if (j >= mp) return;
  double* al = alpha + j * kRmmSMax;
  for (int i = lane; i < kRmmSMax; i += 32) al[i] = 0.0;
  __syncwarp();
  const int s = win.s;
  if (!active[j] || s <= 1) {
    if (lane == 0) al[s - 1] = 1.0;
    return;
  }
  const double* Bj = B + (size_t)j * kRmmSMax * kRmmSMax;
  const int l = win.slot[s - 1];
  const double bll = Bj[l * kRmmSMax + l];
  for (int first = 0; first < s - 1; ++first) {
    const int m = s - 1 - first;  // unknowns: window entries first .. s-2
    double fii = 0.0;
    if (lane < m) {
      const int si = win.slot[first + lane];
      rhs[lane] = -(Bj[si * kRmmSMax + l] - bll);
      for (int k = 0; k < m; ++k) {
        const int sk = win.slot[first + k];
        F[lane][k] = Bj[si * kRmmSMax + sk] - Bj[si * kRmmSMax + l] - Bj[l * kRmmSMax + sk] + bll;
      }
      fii = F[lane][lane];
    }
    // max of the diagonal, in the sequential order
    if (lane == 0) fail = 0;
    __syncwarp();
    double mx = 0.0;
    if (lane == 0) {
      for (int i = 0; i < m; ++i) mx = fmax(mx, F[i][i]);
      if (!(mx > 0.0)) fail = 1;
    }
    (void)fii;
    mx = __shfl_sync(0xffffffffu, mx, 0);
    __syncwarp();
    for (int c = 0; c < m && !fail; ++c) {
      if (lane == c) {
        double piv = F[c][c];
        for (int q = 0; q < c; ++q) piv -= F[c][q] * F[c][q];
        if (!(piv > tol * mx)) fail = 1;
        else F[c][c] = sqrt(piv);
      }
      __syncwarp();
      if (fail) break;
      if (lane > c && lane < m) {
        double t = F[lane][c];
        for (int q = 0; q < c; ++q) t -= F[lane][q] * F[c][q];
        F[lane][c] = t / F[c][c];
      }
      __syncwarp();
    }
    if (fail) {  // drop the oldest entry and retry
      __syncwarp();
      continue;
    }
    if (lane == 0) {
      for (int i = 0; i < m; ++i) {
        double t = rhs[i];
        for (int q = 0; q < i; ++q) t -= F[i][q] * y[q];
        y[i] = t / F[i][i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double t = y[i];
        for (int q = i + 1; q < m; ++q) t -= F[q][i] * y[q];
        y[i] = t / F[i][i];
      }
      double sum = 0.0;
      for (int i = 0; i < m; ++i) {
        al[first + i] = y[i];
        sum += y[i];
      }
      al[s - 1] = 1.0 - sum;
    }
    return;
  }
  if (lane == 0) al[s - 1] = 1.0;  // every difference system singular: keep the newest iterate
}

__global__ void k_rmm_store_gram(double* __restrict__ B, const double* __restrict__ sums, Window win, int slot_new,
                                 int mp) {
  const int j = threadIdx.x;
  if (j >= mp) return;
  double* Bj = B + (size_t)j * kRmmSMax * kRmmSMax;
  const double* sj = sums + (size_t)j * (1 + win.s);
  for (int i = 0; i < win.s; ++i) {
    const int si = win.slot[i];
    Bj[slot_new * kRmmSMax + si] = sj[1 + i];
    Bj[si * kRmmSMax + slot_new] = sj[1 + i];
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
eig_status rmm_combine(const double* xh, const void* rh, const double* thh, const double* alpha, Window win,
                       const double* theta_ref, const int* active, int mp, int64_t n, eig_dtype vt, double* xt,
                       double* hxt, void* rt, double* part, int* nparts, cudaStream_t st) {
  const int grid = rmm_grid(n, mp);
  if (vt == EIG_F32)
    k_rmm_combine<float><<<grid, kRmmThreads, 0, st>>>(xh, (const float*)rh, thh, alpha, win, theta_ref, active, mp,
                                                        n, xt, hxt, (float*)rt, part);
  else
    k_rmm_combine<double><<<grid, kRmmThreads, 0, st>>>(xh, (const double*)rh, thh, alpha, win, theta_ref, active,
                                                         mp, n, xt, hxt, (double*)rt, part);
  EIG_LAUNCH_CHECK("k_rmm_combine");
  *nparts = grid;
  return EIG_OK;
}

eig_status rmm_dots2(const double* xt, const void* rt, const void* hrt, int mp, int64_t n, eig_dtype vt, double* part,
                     int* nparts, cudaStream_t st) {
  const int grid = rmm_grid(n, mp);
  if (vt == EIG_F32)
    k_rmm_dots2<float><<<grid, kRmmThreads, 0, st>>>(xt, (const float*)rt, (const float*)hrt, mp, n, part);
  else
    k_rmm_dots2<double><<<grid, kRmmThreads, 0, st>>>(xt, (const double*)rt, (const double*)hrt, mp, n, part);
  EIG_LAUNCH_CHECK("k_rmm_dots2");
  *nparts = grid;
  return EIG_OK;
}

eig_status rmm_rr2(const double* dots, const int* active, int mp, double* theta, double* g, cudaStream_t st) {
  k_rmm_rr2<<<1, 32, 0, st>>>(dots, active, mp, theta, g);
  EIG_LAUNCH_CHECK("k_rmm_rr2");
  return EIG_OK;
}

eig_status rmm_update(const double* xt, const double* hxt, const void* rt, const void* hrt, const double* g,
                      const double* theta, int slot_new, Window win_after, int mp, int64_t n, eig_dtype vt,
                      double* xh, void* rh, double* thh, double* part, int* nparts, cudaStream_t st) {
  const int grid = rmm_grid(n, mp);
  const size_t sm = (size_t)kRmmThreads * (1 + win_after.s) * 8;
  if (vt == EIG_F32) {
    EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_rmm_update<float>, (int)sm));
    k_rmm_update<float><<<grid, kRmmThreads, sm, st>>>(xt, hxt, (const float*)rt, (const float*)hrt, g, theta,
                                                        slot_new, win_after, mp, n, xh, (float*)rh, thh, part);
  } else {
    EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_rmm_update<double>, (int)sm));
    k_rmm_update<double><<<grid, kRmmThreads, sm, st>>>(xt, hxt, (const double*)rt, (const double*)hrt, g, theta,
                                                         slot_new, win_after, mp, n, xh, (double*)rh, thh, part);
  }
  EIG_LAUNCH_CHECK("k_rmm_update");
  *nparts = grid;
  return EIG_OK;
}

eig_status rmm_start(double* x, const double* hx, const double* num, const double* xnorm2, int mp, int64_t n,
                     eig_dtype vt, int slot, double* xh, void* rh, double* thh, double* theta_out, double* part,
                     int* nparts, cudaStream_t st) {
  const int grid = rmm_grid(n, mp);
  if (vt == EIG_F32)
    k_rmm_start<float><<<grid, kRmmThreads, 0, st>>>(x, hx, num, xnorm2, mp, n, slot, xh, (float*)rh, thh, theta_out,
                                                      part);
  else
    k_rmm_start<double><<<grid, kRmmThreads, 0, st>>>(x, hx, num, xnorm2, mp, n, slot, xh, (double*)rh, thh,
                                                       theta_out, part);
  EIG_LAUNCH_CHECK("k_rmm_start");
  *nparts = grid;
  return EIG_OK;
}

eig_status rmm_diis(const double* B, Window win, const int* active, int mp, double* alpha, cudaStream_t st,
                    double tol) {
  k_rmm_diis<<<mp, 32, 0, st>>>(B, win, active, mp, tol, alpha);
  EIG_LAUNCH_CHECK("k_rmm_diis");
  return EIG_OK;
}

eig_status rmm_store_gram(double* B, const double* sums, Window win_after, int slot_new, int mp, cudaStream_t st) {
  k_rmm_store_gram<<<1, 32, 0, st>>>(B, sums, win_after, slot_new, mp);
  EIG_LAUNCH_CHECK("k_rmm_store_gram");
  return EIG_OK;
}

}  // namespace eig
