// Small dense FP64 kernels, one CTA each: the projected eigenproblems of the Rayleigh-Ritz
// procedure (Eq. rreig; Alg. 1 "solve T U = U Theta"; Alg. 3 "T S = S Theta"), and the
// Cholesky factor of CholeskyQR (Alg. 3).
//
// GB300 runs FP64 at ~1.2 TFLOP/s (about 1/60 of FP32), so the projected problems use an
// O(k^3)-light method instead of Jacobi sweeps: Householder tridiagonalisation, multisection
// bisection on Sturm counts for the wanted (lowest) eigenvalues, inverse iteration for their
// eigenvectors (re-orthogonalised and re-diagonalised inside clusters of close eigenvalues),
// Rayleigh quotients, and back-transformation.  Standard methods: Golub & Van Loan, Matrix
// Computations, Sec. 8.3 (tridiagonalisation), 8.4 (bisection, inverse iteration); Parlett,
// The Symmetric Eigenvalue Problem, Ch. 7.  All work arrays live in a global workspace (a
// few tens of KB, L1/L2 resident).
#include "common.cuh"
#include "small.cuh"

#include <cfloat>

namespace eig {

constexpr int kSmallThreads = 256;

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (lane < nw) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// ---------------------------------------------------------------------------------------
// Householder tridiagonalisation of symmetric a (k x k, row-major, overwritten).
// Reflector j (I - 2 v v^T, unit v, zero in entries <= j) is stored in row j of V.
// ---------------------------------------------------------------------------------------
__device__ void tridiagonalize(double* a, int k, double* d, double* e, double* V, double* p, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  for (int j = 0; j + 2 < k; ++j) {
    const int m0 = j + 1;
    double loc = 0.0;
    for (int i = m0 + tid; i < k; i += nt) loc += a[i * k + j] * a[i * k + j];
    const double s = block_sum(loc, red);
    const double x0 = a[m0 * k + j];
    const double alpha = (s > 0.0) ? -copysign(sqrt(s), x0) : 0.0;
    const double vn2 = 2.0 * s - 2.0 * alpha * x0;
    const bool trivial = !(vn2 > 1e-300);
    const double sc = trivial ? 0.0 : rsqrt(vn2);
    for (int i = tid; i < k; i += nt) {
      double v = 0.0;
      if (i == m0) v = (x0 - alpha) * sc;
      else if (i > m0) v = a[i * k + j] * sc;
      V[j * k + i] = v;
    }
    if (tid == 0) {
      d[j] = a[j * k + j];
      e[j] = trivial ? x0 : alpha;
    }
    __syncthreads();
    if (trivial) continue;
    const double* v = V + j * k;
    // p = A22 v, one warp per row
    for (int i = m0 + w; i < k; i += nw) {
      double acc = 0.0;
      for (int l = m0 + lane; l < k; l += 32) acc += a[i * k + l] * v[l];
      acc = warp_sum(acc);
      if (lane == 0) p[i] = acc;
    }
    __syncthreads();
    loc = 0.0;
    for (int i = m0 + tid; i < k; i += nt) loc += v[i] * p[i];
    const double K = block_sum(loc, red);
    for (int i = m0 + tid; i < k; i += nt) p[i] -= K * v[i];
    __syncthreads();
    const int mm = k - m0;
    for (int idx = tid; idx < mm * mm; idx += nt) {
      const int i = m0 + idx / mm, l = m0 + idx % mm;
      a[i * k + l] -= 2.0 * (v[i] * p[l] + p[i] * v[l]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (k >= 2) {
      d[k - 2] = a[(k - 2) * k + (k - 2)];
      d[k - 1] = a[(k - 1) * k + (k - 1)];
      e[k - 2] = a[(k - 1) * k + (k - 2)];
    } else {
      d[0] = a[0];
    }
  }
  __syncthreads();
}

__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int k, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (q < 0.0) ++c;
  for (int i = 1; i < k; ++i) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = d[i] - x - e2[i - 1] / q;
    if (q < 0.0) ++c;
  }
  return c;
}

// Solve (T - sigma I) y = y in place (tridiagonal T = (d, e)), Gaussian elimination with
// partial pivoting; u0,u1,u2,lm: k-length work arrays; piv: k flags.
__device__ void tri_shift_solve(const double* d, const double* e, int k, double sigma, double tiny, double* u0,
                                double* u1, double* u2, double* lm, unsigned char* piv, double* y) {
  u0[0] = d[0] - sigma;
  u1[0] = (k > 1) ? e[0] : 0.0;
  u2[0] = 0.0;
  for (int i = 0; i + 1 < k; ++i) {
    const double sub = e[i];
    const double nd = d[i + 1] - sigma;
    const double ne = (i + 2 < k) ? e[i + 1] : 0.0;
    if (fabs(u0[i]) >= fabs(sub)) {
      const double piv0 = (u0[i] == 0.0) ? tiny : u0[i];
      const double l = sub / piv0;
      u0[i + 1] = nd - l * u1[i];
      u1[i + 1] = ne - l * u2[i];
      u2[i + 1] = 0.0;
      lm[i] = l;
      piv[i] = 0;
    } else {
      const double l = u0[i] / sub;
      const double t1 = u1[i], t2 = u2[i];
      u0[i] = sub;
      u1[i] = nd;
      u2[i] = ne;
      u0[i + 1] = t1 - l * nd;
      u1[i + 1] = t2 - l * ne;
      u2[i + 1] = 0.0;
      lm[i] = l;
      piv[i] = 1;
    }
  }
  for (int i = 0; i < k; ++i)
    if (fabs(u0[i]) < tiny) u0[i] = copysign(tiny, u0[i] == 0.0 ? 1.0 : u0[i]);
  for (int i = 0; i + 1 < k; ++i) {
    if (piv[i]) {
      const double t = y[i];
      y[i] = y[i + 1];
      y[i + 1] = t;
    }
    y[i + 1] -= lm[i] * y[i];
  }
  y[k - 1] /= u0[k - 1];
  if (k > 1) y[k - 2] = (y[k - 2] - u1[k - 2] * y[k - 1]) / u0[k - 2];
  for (int i = k - 3; i >= 0; --i) y[i] = (y[i] - u1[i] * y[i + 1] - u2[i] * y[i + 2]) / u0[i];
}

__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (double)(h & 0xFFFFFF) / 8388608.0 - 1.0;  // in [-1, 1)
}

// Tridiagonal T y = theta y for the lowest m eigenpairs.  Y (k x m, column t contiguous at
// Y + t*k) receives unit eigenvectors, w the eigenvalues (ascending).
struct TriWork {
  double *d, *e, *e2, *u0, *u1, *u2, *lm, *Y, *P;  // u*, lm: m*k each; Y: m*k; P: 32*32
  unsigned char* piv;                              // m*k
  double* lo;                                      // m
  double* hi;                                      // m
  int* cnt;                                        // nt
};

__device__ void tri_eig_lowest(int k, int m, TriWork W, double* w, double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // squared off-diagonals, Gershgorin bounds, norm
  double glo = DBL_MAX, ghi = -DBL_MAX, mx = 0.0, me2 = 0.0;
  for (int i = tid; i < k; i += nt) {
    const double el = (i > 0) ? fabs(W.e[i - 1]) : 0.0, er = (i + 1 < k) ? fabs(W.e[i]) : 0.0;
    glo = fmin(glo, W.d[i] - el - er);
    ghi = fmax(ghi, W.d[i] + el + er);
    mx = fmax(mx, fabs(W.d[i]) + el + er);
    if (i + 1 < k) { W.e2[i] = W.e[i] * W.e[i]; me2 = fmax(me2, W.e2[i]); }
  }
  glo = -block_max(-glo, red);
  ghi = block_max(ghi, red);
  const double tnorm = fmax(block_max(mx, red), 1e-300);
  me2 = block_max(me2, red);
  const double pivmin = 1e-290 * fmax(1.0, me2);
  glo -= 2.0 * DBL_EPSILON * tnorm + 1e-300;
  ghi += 2.0 * DBL_EPSILON * tnorm + 1e-300;
  // multisection: G threads per wanted eigenvalue
  const int G = max(1, nt / m);
  for (int t = tid; t < m; t += nt) { W.lo[t] = glo; W.hi[t] = ghi; }
  __syncthreads();
  const int rounds = (int)ceil(56.0 / log2((double)G + 1.0)) + 1;
  for (int r = 0; r < rounds; ++r) {
    const int t = tid / G, g = tid % G;
    if (t < m) {
      const double lo = W.lo[t], hi = W.hi[t];
      const double x = lo + (hi - lo) * (double)(g + 1) / (double)(G + 1);
      W.cnt[tid] = sturm_count(W.d, W.e2, k, x, pivmin);
    }
    __syncthreads();
    if (tid < m) {
      const double lo = W.lo[tid], hi = W.hi[tid];
      double nlo = lo, nhi = hi;
      for (int gg = 0; gg < G; ++gg) {
        const double x = lo + (hi - lo) * (double)(gg + 1) / (double)(G + 1);
        if (W.cnt[tid * G + gg] <= tid) nlo = x;
        else { nhi = x; break; }
      }
      W.lo[tid] = nlo;
      W.hi[tid] = nhi;
    }
    __syncthreads();
  }
  // inverse iteration, one thread per eigenvector, distinct pseudo-random starts
  const double tiny = fmax(DBL_EPSILON * tnorm, 1e-280);
  for (int t = tid; t < m; t += nt) {
    const double lam = 0.5 * (W.lo[t] + W.hi[t]);
    double* y = W.Y + (size_t)t * k;
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) { y[i] = hash_unit(t + 1, i + 1); nrm += y[i] * y[i]; }
    nrm = rsqrt(nrm);
    for (int i = 0; i < k; ++i) y[i] *= nrm;
    for (int it = 0; it < 3; ++it) {
      tri_shift_solve(W.d, W.e, k, lam, tiny, W.u0 + (size_t)t * k, W.u1 + (size_t)t * k, W.u2 + (size_t)t * k,
                      W.lm + (size_t)t * k, W.piv + (size_t)t * k, y);
      // scale by the largest entry first: the solve can grow y by up to 1/tiny
      double mx = 0.0;
      for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(y[i]));
      if (!(mx > 0.0) || !isfinite(mx)) {
        for (int i = 0; i < k; ++i) y[i] = (i == t % k) ? 1.0 : 0.0;
        break;
      }
      nrm = 0.0;
      for (int i = 0; i < k; ++i) { y[i] /= mx; nrm += y[i] * y[i]; }
      nrm = rsqrt(nrm);
      for (int i = 0; i < k; ++i) y[i] *= nrm;
    }
    w[t] = lam;
  }
  __syncthreads();
  // clusters of close eigenvalues: MGS (warp 0), then diagonalise the projected cluster block
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double ctol = 1e-3 * tnorm;
    int cs = 0;
    for (int t = 1; t <= m; ++t) {
      const bool brk = (t == m) || (w[t] - w[t - 1] > ctol);
      if (!brk) continue;
      const int c = t - cs;
      if (c > 1) {
        for (int a = cs; a < t; ++a) {
          double* ya = W.Y + (size_t)a * k;
          for (int pass = 0; pass < 2; ++pass) {
            for (int b = cs; b < a; ++b) {
              const double* yb = W.Y + (size_t)b * k;
              double dt = 0.0;
              for (int i = lane; i < k; i += 32) dt += ya[i] * yb[i];
              dt = warp_sum(dt);
              for (int i = lane; i < k; i += 32) ya[i] -= dt * yb[i];
              __syncwarp();
            }
          }
          double nn = 0.0;
          for (int i = lane; i < k; i += 32) nn += ya[i] * ya[i];
          nn = rsqrt(fmax(warp_sum(nn), 1e-300));
          for (int i = lane; i < k; i += 32) ya[i] *= nn;
          __syncwarp();
        }
        if (c <= 32) {
          // projected block P = Yc^T T Yc (c x c)
          for (int a = 0; a < c; ++a) {
            const double* ya = W.Y + (size_t)(cs + a) * k;
            for (int b = 0; b <= a; ++b) {
              const double* yb = W.Y + (size_t)(cs + b) * k;
              double s = 0.0;
              for (int i = lane; i < k; i += 32) {
                double ty = W.d[i] * yb[i];
                if (i > 0) ty += W.e[i - 1] * yb[i - 1];
                if (i + 1 < k) ty += W.e[i] * yb[i + 1];
                s += ya[i] * ty;
              }
              s = warp_sum(s);
              if (lane == 0) { W.P[a * 32 + b] = s; W.P[b * 32 + a] = s; }
            }
          }
          __syncwarp();
          // cyclic Jacobi on P (lane 0), rotations applied to the cluster vectors by the warp
          for (int sweep = 0; sweep < 30; ++sweep) {
            double off = 0.0;
            if (lane == 0)
              for (int a = 0; a < c; ++a)
                for (int b = 0; b < a; ++b) off += W.P[a * 32 + b] * W.P[a * 32 + b];
            off = __shfl_sync(0xffffffffu, off, 0);
            if (off < 1e-30 * tnorm * tnorm) break;
            for (int a = 0; a < c; ++a) {
              for (int b = a + 1; b < c; ++b) {
                double cth = 1.0, sth = 0.0;
                if (lane == 0) {
                  const double apq = W.P[a * 32 + b];
                  if (fabs(apq) > 1e-300) {
                    const double tau = (W.P[b * 32 + b] - W.P[a * 32 + a]) / (2.0 * apq);
                    const double tt = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    cth = rsqrt(1.0 + tt * tt);
                    sth = tt * cth;
                    for (int r2 = 0; r2 < c; ++r2) {
                      const double pa = W.P[r2 * 32 + a], pb = W.P[r2 * 32 + b];
                      W.P[r2 * 32 + a] = cth * pa - sth * pb;
                      W.P[r2 * 32 + b] = sth * pa + cth * pb;
                    }
                    for (int r2 = 0; r2 < c; ++r2) {
                      const double pa = W.P[a * 32 + r2], pb = W.P[b * 32 + r2];
                      W.P[a * 32 + r2] = cth * pa - sth * pb;
                      W.P[b * 32 + r2] = sth * pa + cth * pb;
                    }
                  }
                }
                cth = __shfl_sync(0xffffffffu, cth, 0);
                sth = __shfl_sync(0xffffffffu, sth, 0);
                if (sth != 0.0) {
                  double* ya = W.Y + (size_t)(cs + a) * k;
                  double* yb = W.Y + (size_t)(cs + b) * k;
                  for (int i = lane; i < k; i += 32) {
                    const double va = ya[i], vb = yb[i];
                    ya[i] = cth * va - sth * vb;
                    yb[i] = sth * va + cth * vb;
                  }
                }
                __syncwarp();
              }
            }
          }
          // sort the cluster ascending (selection sort on P's diagonal, swap vectors)
          for (int a = 0; a < c; ++a) {
            int best = a;
            double bv = W.P[a * 32 + a];
            for (int b = a + 1; b < c; ++b)
              if (W.P[b * 32 + b] < bv) { bv = W.P[b * 32 + b]; best = b; }
            if (best != a) {
              double* ya = W.Y + (size_t)(cs + a) * k;
              double* yb = W.Y + (size_t)(cs + best) * k;
              for (int i = lane; i < k; i += 32) { const double tv = ya[i]; ya[i] = yb[i]; yb[i] = tv; }
              __syncwarp();
              if (lane == 0) {
                const double tv = W.P[a * 32 + a];
                W.P[a * 32 + a] = W.P[best * 32 + best];
                W.P[best * 32 + best] = tv;
              }
              __syncwarp();
            }
          }
        }
      }
      cs = t;
    }
  }
  __syncthreads();
  // Rayleigh quotients give the final eigenvalues
  for (int t = tid; t < m; t += nt) {
    const double* y = W.Y + (size_t)t * k;
    double s = 0.0;
    for (int i = 0; i < k; ++i) {
      double ty = W.d[i] * y[i];
      if (i > 0) ty += W.e[i - 1] * y[i - 1];
      if (i + 1 < k) ty += W.e[i] * y[i + 1];
      s += y[i] * ty;
    }
    w[t] = s;
  }
  __syncthreads();
  // keep ascending order (clusters may reorder neighbours by roundoff): insertion sort by thread 0
  if (tid == 0) {
    for (int a = 1; a < m; ++a) {
      int b = a;
      while (b > 0 && w[b - 1] > w[b]) {
        const double tv = w[b]; w[b] = w[b - 1]; w[b - 1] = tv;
        double* ya = W.Y + (size_t)b * k;
        double* yb = W.Y + (size_t)(b - 1) * k;
        for (int i = 0; i < k; ++i) { const double tt = ya[i]; ya[i] = yb[i]; yb[i] = tt; }
        --b;
      }
    }
  }
  __syncthreads();
}

// Z (k x m row-major) = Q Y with Q = H_0 H_1 ... H_{k-3}; Y column t at Y + t*k.
__device__ void back_transform(int k, int m, const double* V, double* Y, double* Z) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = w; t < m; t += nw) {
    double* y = Y + (size_t)t * k;
    for (int j = k - 3; j >= 0; --j) {
      const double* v = V + (size_t)j * k;
      double dt = 0.0;
      for (int i = j + 1 + lane; i < k; i += 32) dt += v[i] * y[i];
      dt = warp_sum(dt);
      for (int i = j + 1 + lane; i < k; i += 32) y[i] -= 2.0 * dt * v[i];
      __syncwarp();
    }
    for (int i = lane; i < k; i += 32) Z[(size_t)i * m + t] = y[i];
  }
  __syncthreads();
}

// Workspace layout for a k x k problem with m wanted pairs.
struct SyevLayout {
  size_t a, V, p, d, e, e2, u0, u1, u2, lm, Y, P, lo, hi, cnt, piv, total;
  SyevLayout(int k, int m) {
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
    a = take((size_t)k * k * 8); V = take((size_t)k * k * 8); p = take((size_t)k * 8);
    d = take((size_t)k * 8); e = take((size_t)k * 8); e2 = take((size_t)k * 8);
    u0 = take((size_t)m * k * 8); u1 = take((size_t)m * k * 8); u2 = take((size_t)m * k * 8);
    lm = take((size_t)m * k * 8); Y = take((size_t)m * k * 8); P = take(32 * 32 * 8);
    lo = take((size_t)m * 8); hi = take((size_t)m * 8); cnt = take(kSmallThreads * 4);
    piv = take((size_t)m * k);
    total = o;
  }
};

__device__ TriWork make_triwork(unsigned char* base, const SyevLayout& L) {
  TriWork W;
  W.d = (double*)(base + L.d); W.e = (double*)(base + L.e); W.e2 = (double*)(base + L.e2);
  W.u0 = (double*)(base + L.u0); W.u1 = (double*)(base + L.u1); W.u2 = (double*)(base + L.u2);
  W.lm = (double*)(base + L.lm); W.Y = (double*)(base + L.Y); W.P = (double*)(base + L.P);
  W.lo = (double*)(base + L.lo); W.hi = (double*)(base + L.hi); W.cnt = (int*)(base + L.cnt);
  W.piv = base + L.piv;
  return W;
}

// Eigen-decomposition of the symmetric matrix already in L.a (workspace); lowest m.
__device__ void syev_in_work(unsigned char* base, const SyevLayout& L, int k, int m, double* w, double* Z,
                             double* red) {
  double* a = (double*)(base + L.a);
  double* V = (double*)(base + L.V);
  double* p = (double*)(base + L.p);
  TriWork W = make_triwork(base, L);
  if (k == 1) {
    if (threadIdx.x == 0) { w[0] = a[0]; Z[0] = 1.0; }
    __syncthreads();
    return;
  }
  tridiagonalize(a, k, W.d, W.e, V, p, red);
  tri_eig_lowest(k, m, W, w, red);
  back_transform(k, m, V, W.Y, Z);
}

__global__ void __launch_bounds__(kSmallThreads) k_small_syev(const double* A, int k, int m, double* w, double* Z,
                                                              unsigned char* work, SyevLayout L, int* info) {
  __shared__ double red[33];
  double* a = (double*)(work + L.a);
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
    const int r = i / k, c = i % k;
    a[i] = 0.5 * (A[r * k + c] + A[c * k + r]);
  }
  __syncthreads();
  syev_in_work(work, L, k, m, w, Z, red);
  if (threadIdx.x == 0 && info) *info = SMALL_OK;
}

size_t small_syev_work_bytes(int k, int m) { return SyevLayout(k, m).total; }

// Tridiagonal input (Lanczos T_k of Eq. lanfac): lowest m eigenpairs of (d, e), Z (k x m).
__global__ void __launch_bounds__(kSmallThreads) k_small_tri_eig(const double* d, const double* e, int k, int m,
                                                                 double* w, double* Z, unsigned char* work,
                                                                 SyevLayout L) {
  __shared__ double red[33];
  TriWork W = make_triwork(work, L);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    W.d[i] = d[i];
    W.e[i] = (i + 1 < k) ? e[i] : 0.0;
  }
  __syncthreads();
  if (k == 1) {
    if (threadIdx.x == 0) { w[0] = W.d[0]; Z[0] = 1.0; }
    return;
  }
  tri_eig_lowest(k, m, W, w, red);
  for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
    const int i = idx / m, t = idx % m;
    Z[idx] = W.Y[(size_t)t * k + i];
  }
}

eig_status small_tri_eig(const double* d, const double* e, int k, int m, double* w, double* Z, void* work,
                         cudaStream_t st) {
  if (k < 1 || m < 1 || m > k || m > 256) return EIG_EINVAL;
  SyevLayout L(k, m);
  k_small_tri_eig<<<1, kSmallThreads, 0, st>>>(d, e, k, m, w, Z, (unsigned char*)work, L);
  EIG_LAUNCH_CHECK("k_small_tri_eig");
  return EIG_OK;
}

eig_status small_syev(const double* A, int k, int m, double* w, double* Z, void* work, int* info, cudaStream_t st) {
  if (k < 1 || m < 1 || m > k || k > kSmallMax || m > 256) return EIG_EINVAL;
  SyevLayout L(k, m);
  k_small_syev<<<1, kSmallThreads, 0, st>>>(A, k, m, w, Z, (unsigned char*)work, L, info);
  EIG_LAUNCH_CHECK("k_small_syev");
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// Cholesky (lower, in place) of a k x k SPD matrix g; breakdown when a pivot <= piv_tol.
// Returns SMALL_OK / SMALL_BREAKDOWN (uniform across the CTA).
// ---------------------------------------------------------------------------------------
__device__ int cholesky_lower(double* g, int k, double piv_tol, int* flag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *flag = SMALL_OK;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const double piv = g[j * k + j];
    if (!(piv > piv_tol)) {
      if (tid == 0) *flag = SMALL_BREAKDOWN;
      __syncthreads();
      return SMALL_BREAKDOWN;
    }
    const double ljj = sqrt(piv);
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += nt) g[i * k + j] /= ljj;
    __syncthreads();
    if (tid == 0) g[j * k + j] = ljj;
    const int mm = k - j - 1;
    for (int idx = tid; idx < mm * mm; idx += nt) {
      const int i = j + 1 + idx / mm, l = j + 1 + idx % mm;
      if (l <= i) g[i * k + l] -= g[i * k + j] * g[l * k + j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    if (l > i) g[idx] = 0.0;
  }
  __syncthreads();
  return SMALL_OK;
}

// Rayleigh-Ritz on (A, G), see small.cuh.
struct RRLayout {
  size_t g, dsc, t, syev, z, total;
  SyevLayout S;
  RRLayout(int k, int nb) : S(k, nb) {
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~size_t(255); return r; };
    g = take((size_t)k * k * 8); dsc = take((size_t)k * 8); t = take((size_t)k * k * 8);
    z = take((size_t)k * nb * 8);
    syev = take(S.total);
    total = o;
  }
};

__global__ void __launch_bounds__(kSmallThreads) k_small_rr(const double* A, const double* G, int k, int nb,
                                                            double piv_tol, int pivoted, double* theta, double* C,
                                                            float* C32, unsigned char* work, RRLayout L, int* info) {
  __shared__ double red[33];
  __shared__ int flag;
  __shared__ int sel[kSmallMax / 4];
  __shared__ int ksel, pstar;
  __shared__ double dstar;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* g = (double*)(work + L.g);
  double* dsc = (double*)(work + L.dsc);
  double* t = (double*)(work + L.t);
  double* z = (double*)(work + L.z);
  unsigned char* sw = work + L.syev;
  double* a = (double*)(sw + L.S.a);
  // column scaling to a unit-diagonal Gram
  for (int i = tid; i < k; i += nt) {
    const double gi = G[i * k + i];
    dsc[i] = (gi > 0.0) ? rsqrt(gi) : 0.0;
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    g[idx] = 0.5 * (G[i * k + l] + G[l * k + i]) * dsc[i] * dsc[l];
    t[idx] = 0.5 * (A[i * k + l] + A[l * k + i]) * dsc[i] * dsc[l];
  }
  __syncthreads();
  int kk = k;
  if (pivoted) {
    // rank-revealing (diagonally pivoted) Cholesky of the scaled Gram on a copy in a: the
    // basis columns are taken by largest remaining pivot until it falls to piv_tol; the
    // Rayleigh-Ritz below then runs on those columns only
    for (int idx = tid; idx < k * k; idx += nt) a[idx] = g[idx];
    if (tid == 0) ksel = 0;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
      if (tid == 0) {
        int best = -1;
        double bd = -1.0;
        for (int i = 0; i < k; ++i)   // taken columns carry -1 on the diagonal
          if (a[i * k + i] > bd) { bd = a[i * k + i]; best = i; }
        pstar = (best >= 0 && bd > piv_tol) ? best : -1;
        dstar = bd;
        if (pstar >= 0) sel[ksel] = pstar;
      }
      __syncthreads();
      if (pstar < 0) break;
      const int p = pstar;
      const double rp = rsqrt(dstar);
      // Schur complement over the columns not yet taken (the taken ones are never read again)
      for (int idx = tid; idx < k * k; idx += nt) {
        const int i = idx / k, l = idx % k;
        if (i != p && l != p) a[idx] -= (a[i * k + p] * rp) * (a[l * k + p] * rp);
      }
      __syncthreads();
      if (tid == 0) {
        for (int i = 0; i < k; ++i) { a[i * k + p] = 0.0; a[p * k + i] = 0.0; }
        a[p * k + p] = -1.0;   // taken
        ++ksel;
      }
      __syncthreads();
    }
    kk = ksel;
    if (kk < nb) {
      if (tid == 0) *info = SMALL_BREAKDOWN;
      return;
    }
    // compact g, t (and the scaling) to the kk taken columns, in the order taken
    for (int idx = tid; idx < kk * kk; idx += nt) a[idx] = g[sel[idx / kk] * k + sel[idx % kk]];
    __syncthreads();
    for (int idx = tid; idx < kk * kk; idx += nt) g[idx] = a[idx];
    __syncthreads();
    for (int idx = tid; idx < kk * kk; idx += nt) a[idx] = t[sel[idx / kk] * k + sel[idx % kk]];
    __syncthreads();
    for (int idx = tid; idx < kk * kk; idx += nt) t[idx] = a[idx];
    for (int i = tid; i < kk; i += nt) z[i] = dsc[sel[i]];
    __syncthreads();
    for (int i = tid; i < kk; i += nt) dsc[i] = z[i];
    __syncthreads();
  }
  if (cholesky_lower(g, kk, piv_tol, &flag) != SMALL_OK) {
    if (tid == 0) *info = SMALL_BREAKDOWN;
    return;
  }
  // W = L^{-1} T (forward substitution per column, thread per column) -> stored in a
  for (int c = tid; c < kk; c += nt) {
    for (int i = 0; i < kk; ++i) {
      double s = t[i * kk + c];
      for (int l = 0; l < i; ++l) s -= g[i * kk + l] * a[l * kk + c];
      a[i * kk + c] = s / g[i * kk + i];
    }
  }
  __syncthreads();
  // T = L^{-1} W^T  (columns of W^T are rows of W) -> t
  for (int c = tid; c < kk; c += nt) {
    for (int i = 0; i < kk; ++i) {
      double s = a[c * kk + i];
      for (int l = 0; l < i; ++l) s -= g[i * kk + l] * t[l * kk + c];
      t[i * kk + c] = s / g[i * kk + i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kk * kk; idx += nt) {
    const int i = idx / kk, l = idx % kk;
    a[idx] = 0.5 * (t[i * kk + l] + t[l * kk + i]);
  }
  __syncthreads();
  syev_in_work(sw, L.S, kk, nb, theta, z, red);
  // C = D L^{-T} Z (backward substitution per column)
  for (int c = tid; c < nb; c += nt) {
    for (int i = kk - 1; i >= 0; --i) {
      double s = z[i * nb + c];
      for (int l = i + 1; l < kk; ++l) s -= g[l * kk + i] * C[l * nb + c];
      C[i * nb + c] = s / g[i * kk + i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < kk * nb; idx += nt) C[idx] *= dsc[idx / nb];
  __syncthreads();
  if (pivoted) {
    // rows of the taken columns back to their basis positions, zero rows for the others
    for (int idx = tid; idx < kk * nb; idx += nt) z[idx] = C[idx];
    __syncthreads();
    for (int idx = tid; idx < k * nb; idx += nt) C[idx] = 0.0;
    __syncthreads();
    for (int idx = tid; idx < kk * nb; idx += nt) C[sel[idx / nb] * nb + idx % nb] = z[idx];
    __syncthreads();
  }
  if (C32)
    for (int idx = tid; idx < k * nb; idx += nt) C32[idx] = (float)C[idx];
  if (tid == 0) *info = SMALL_OK;
}

size_t small_rr_work_bytes(int k, int nb) { return RRLayout(k, nb).total; }

eig_status small_rr(const double* A, const double* G, int k, int nb, double piv_tol, double* theta, double* C,
                    float* C32, void* work, int* info, cudaStream_t st, int pivoted) {
  if (k < 1 || nb < 1 || nb > k || k > kSmallMax * 4) return EIG_EINVAL;
  if (pivoted && k > kSmallMax / 4) return EIG_EINVAL;
  RRLayout L(k, nb);
  k_small_rr<<<1, kSmallThreads, 0, st>>>(A, G, k, nb, piv_tol, pivoted, theta, C, C32, (unsigned char*)work, L,
                                          info);
  EIG_LAUNCH_CHECK("k_small_rr");
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// CholQR factor: G = R^T R, R upper, Rinv = R^{-1}
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSmallThreads) k_small_chol_inv(const double* G, int k, double piv_tol, double* R,
                                                                  double* Rinv, float* Rinv32, double* work,
                                                                  int* info) {
  __shared__ int flag;
  __shared__ double red[33];
  const int tid = threadIdx.x, nt = blockDim.x;
  double* g = work;  // k*k lower factor
  double md = 0.0;
  for (int i = tid; i < k; i += nt) md = fmax(md, G[i * k + i]);
  md = block_max(md, red);
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    g[idx] = 0.5 * (G[i * k + l] + G[l * k + i]);
  }
  __syncthreads();
  if (cholesky_lower(g, k, piv_tol * md, &flag) != SMALL_OK) {
    if (tid == 0) *info = SMALL_BREAKDOWN;
    return;
  }
  // R = L^T; Rinv = (L^{-1})^T: column c of L^{-1} by forward substitution (thread per column)
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    R[idx] = (l >= i) ? g[l * k + i] : 0.0;
  }
  for (int c = tid; c < k; c += nt) {
    for (int i = 0; i < k; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) s -= g[i * k + l] * Rinv[c * k + l];   // Linv[l][c] stored as Rinv[c][l]
      Rinv[c * k + i] = (i < c) ? 0.0 : s / g[i * k + i];
    }
  }
  __syncthreads();
  // Rinv[c][i] currently holds Linv[i][c] = (Linv^T)[c][i] = Rinv[c][i]: already upper triangular
  for (int idx = tid; idx < k * k; idx += nt) {
    if (Rinv32) Rinv32[idx] = (float)Rinv[idx];
  }
  if (tid == 0) *info = SMALL_OK;
}

eig_status small_chol_inv(const double* G, int k, double piv_tol, double* R, double* Rinv, float* Rinv32, void* work,
                          int* info, cudaStream_t st) {
  if (k < 1 || k > kSmallMax * 4) return EIG_EINVAL;
  k_small_chol_inv<<<1, kSmallThreads, 0, st>>>(G, k, piv_tol, R, Rinv, Rinv32, (double*)work, info);
  EIG_LAUNCH_CHECK("k_small_chol_inv");
  return EIG_OK;
}

}  // namespace eig
