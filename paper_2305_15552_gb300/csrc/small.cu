// Small dense kernels in FP64-equivalent (double-float) arithmetic, one CTA each: the projected
// eigenproblems of the Rayleigh-Ritz
// procedure (Eq. rreig; Alg. 1 "solve T U = U Theta"; Alg. 3 "T S = S Theta"), and the
// Cholesky factor of CholeskyQR (Alg. 3).
//
// GB300 runs FP64 at ~1.2 TFLOP/s (about 1/60 of FP32; a dependent FP64 multiply-add takes
// ~64 cycles, a divide ~420), so these sequential solves compute in double-float (pairs of
// FP32, ~2^-46 relative, dfloat.cuh) with inputs and outputs in FP64, and the projected
// problems use an O(k^3)-light method instead of Jacobi sweeps: Householder tridiagonalisation, multisection
// bisection on Sturm counts for the wanted (lowest) eigenvalues, inverse iteration for their
// eigenvectors (re-orthogonalised and re-diagonalised inside clusters of close eigenvalues),
// Rayleigh quotients, and back-transformation.  Standard methods: Golub & Van Loan, Matrix
// Computations, Sec. 8.3 (tridiagonalisation), 8.4 (bisection, inverse iteration); Parlett,
// The Symmetric Eigenvalue Problem, Ch. 7.  All work arrays live in dynamic shared memory when
// they fit (every k up to ~60 with its wanted pairs), else in a global workspace.
#include "common.cuh"
#include "dfloat.cuh"
#include "small.cuh"

#include <cfloat>

namespace eig {

constexpr int kSmallThreads = 512;
// Scalar type of the small solvers: double-float (FP32 pairs), whose dependent operations GB300
// runs an order of magnitude faster than its FP64 ones at ~2^-46 relative precision.
typedef dfl SmallR;
// Workspaces up to this size live in dynamic shared memory (every access of the sequential
// phases then costs a shared-memory, not an L1/L2, round trip); larger ones stay in the
// caller's global workspace.
constexpr size_t kSmallSmemBytes = 200 * 1024;

// Warp and CTA reductions for the scalar type R (FP64 or double-float); red: 33 scalars of
// shared memory.
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor(v, o);
  return v;
}

template <typename R>
__device__ R block_sum(R v, R* red) {
  v = wsum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    R t = (lane < nw) ? red[lane] : R(0.0);
    t = wsum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

template <typename R>
__device__ R block_max(R v, R* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, shfl_xor(v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    R t = (lane < nw) ? red[lane] : R(0.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, shfl_xor(t, o));
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// ---------------------------------------------------------------------------------------
// Householder tridiagonalisation of symmetric a (k x k, row-major, overwritten).
// Reflector j (I - 2 v v^T, unit v, zero in entries <= j) is stored in row j of V.
// ---------------------------------------------------------------------------------------

// Reflector of column j from the current a, computed by one warp (lanes stride the rows):
// V row j, d[j], e[j]; returns whether the column is already reduced (no reflection).
template <typename R>
__device__ __forceinline__ bool householder_column(const R* a, int k, int j, R* d, R* e, R* V, int lane) {
  const int m0 = j + 1;
  R loc = 0.0;
  for (int i = m0 + lane; i < k; i += 32) loc = dfma(a[i * k + j], a[i * k + j], loc);
  const R s = wsum(loc);
  const R x0 = a[m0 * k + j];
  const R alpha = (s > R(0.0)) ? -copysign(sqrt(s), x0) : R(0.0);
  const R vn2 = R(2.0) * s - R(2.0) * alpha * x0;
  const bool trivial = !(vn2 > R(SmallTraits<R>::floor));
  const R sc = trivial ? R(0.0) : rsqrt(vn2);
  R* v = V + j * k;
  for (int i = lane; i < k; i += 32) v[i] = (i == m0) ? (x0 - alpha) * sc : (i > m0 ? a[i * k + j] * sc : R(0.0));
  if (lane == 0) {
    d[j] = a[j * k + j];
    e[j] = trivial ? x0 : alpha;
  }
  return trivial;
}

// Two CTA barriers per reflector (after p = A v, after the update).  Look-ahead: warp 0
// updates column j + 1 first and computes the next reflector from it while the other warps
// update the rest of the trailing block.  Every warp reduces v^T p by itself.
template <typename R>
__device__ void tridiagonalize(R* a, int k, R* d, R* e, R* V, R* p, R* vp) {
  __shared__ int s_triv[2];   // flag of reflector j in s_triv[j & 1] (read after a barrier,
                              // rewritten only after the next one)
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  bool triv = false;
  if (k >= 3) {
    if (warp == 0) {
      const bool t0 = householder_column(a, k, 0, d, e, V, lane);
      if (lane == 0) s_triv[0] = t0;
    }
    __syncthreads();
    triv = s_triv[0];
  }
  for (int j = 0; j + 2 < k; ++j) {
    const int m0 = j + 1, rows = k - m0;
    const bool next = j + 3 < k;   // a reflector follows this one
    if (triv) {                    // uniform: nothing of a changes; the next column as it is
      if (next) {
        if (warp == 0) {
          const bool t1 = householder_column(a, k, j + 1, d, e, V, lane);
          if (lane == 0) s_triv[(j + 1) & 1] = t1;
        }
        __syncthreads();
        triv = s_triv[(j + 1) & 1];
      }
      continue;
    }
    const R* v = V + j * k;
    // p = A22 v and v_i p_i: eight consecutive lanes per row, two partial sums each
    for (int base = 0; base < rows * 8; base += nt) {
      const int idx = base + tid;
      const bool act = idx < rows * 8;
      const int i = m0 + (act ? idx >> 3 : 0), q = idx & 7;
      R acc = 0.0, acc2 = 0.0;
      if (act) {
        int l = m0 + q;
        for (; l + 8 < k; l += 16) {
          acc = dfma(a[i * k + l], v[l], acc);
          acc2 = dfma(a[i * k + l + 8], v[l + 8], acc2);
        }
        if (l < k) acc = dfma(a[i * k + l], v[l], acc);
      }
      acc = acc + acc2;
      acc = acc + shfl_xor(acc, 1);
      acc = acc + shfl_xor(acc, 2);
      acc = acc + shfl_xor(acc, 4);
      if (act && q == 0) {
        p[i] = acc;
        vp[i] = v[i] * acc;
      }
    }
    __syncthreads();
    R loc = 0.0;
    for (int i = m0 + lane; i < k; i += 32) loc += vp[i];
    const R K = wsum(loc);
    // A22 <- A22 - 2 (v w^T + w v^T), w = p - (v^T p) v, on the lower triangle (each element
    // stored to both halves)
    if (warp == 0) {
      // column m0 (and row m0), then the next reflector
      const R vm = v[m0];
      const R wm = dfma(-K, vm, p[m0]);
      for (int i = m0 + lane; i < k; i += 32) {
        const R vi = v[i];
        const R r0 = dfma(R(-2.0), dfma(vi, wm, dfma(-K, vi, p[i]) * vm), a[i * k + m0]);
        a[i * k + m0] = r0;
        a[m0 * k + i] = r0;
      }
      __syncwarp();
      if (next) {
        const bool t1 = householder_column(a, k, j + 1, d, e, V, lane);
        if (lane == 0) s_triv[(j + 1) & 1] = t1;
      }
    } else {
      // the rest: thread (ti, tc) of a ((nt - 32)/16) x 16 grid takes rows m0 + 1 + ti + nr s
      // and columns m0 + 1 + tc + 16 u
      const int t2 = tid - 32, tc = t2 & 15, ti = t2 >> 4, nr = (nt - 32) >> 4;
      for (int i = m0 + 1 + ti; i < k; i += nr) {
        const R vi = v[i];
        const R wi = dfma(-K, vi, p[i]);
        int l = m0 + 1 + tc;
        for (; l + 16 <= i; l += 32) {
          const R a0 = a[i * k + l], a1 = a[i * k + l + 16];
          const R vl0 = v[l], vl1 = v[l + 16], pl0 = p[l], pl1 = p[l + 16];
          const R r0 = dfma(R(-2.0), dfma(vi, dfma(-K, vl0, pl0), wi * vl0), a0);
          const R r1 = dfma(R(-2.0), dfma(vi, dfma(-K, vl1, pl1), wi * vl1), a1);
          a[i * k + l] = r0; a[l * k + i] = r0;
          a[i * k + l + 16] = r1; a[(l + 16) * k + i] = r1;
        }
        if (l <= i) {
          const R vl = v[l];
          const R r0 = dfma(R(-2.0), dfma(vi, dfma(-K, vl, p[l]), wi * vl), a[i * k + l]);
          a[i * k + l] = r0; a[l * k + i] = r0;
        }
      }
    }
    __syncthreads();
    if (next) triv = s_triv[(j + 1) & 1];
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

// Number of eigenvalues of the tridiagonal (d, e2 = e^2) below x: the sign changes of the
// leading principal minors p_i = (d_i - x) p_{i-1} - e2_{i-1} p_{i-2} (Sturm sequence, Golub &
// Van Loan Sec. 8.4.1).  This division-free form has the ratio form's backward stability
// (p_i / p_{i-1} is the LDL^T pivot, and each operation's rounding is a relative perturbation
// of d_i - x or e2_{i-1}); the pair (p_{i-1}, p_i) is rescaled by powers of two, exactly, to
// stay in range (the matrix is scaled to norm <= 1, so a step grows |p| by at most 3x).  A
// zero minor counts as a sign change (an eigenvalue at x is counted below it).
template <typename R>
__device__ __forceinline__ int sturm_count(const R* __restrict__ d, const R* __restrict__ e2, int k, R x) {
  R pm = 1.0, pc = d[0] - x;
  if (lead_f32(pc) == 0.0f) pc = R(-0x1p-40);
  int c = sign_bit(pc);
  for (int i = 1; i < k; ++i) {
    const R t = e2[i - 1] * pm;
    const R pn = dfma(d[i] - x, pc, -t);
    pm = pc;
    pc = (lead_f32(pn) == 0.0f) ? -scale2(pm, -40) : pn;
    c += sign_bit(pc) ^ sign_bit(pm);
    // every step: a run of tiny pivots (a graded matrix) shrinks p without bound, so the
    // pair is kept in [2^-64, 2^64]; a minor that still underflows is a pivot below ~2^-62 of
    // the norm, counted as zero (the count of a matrix perturbed that little)
    const float big = fmaxf(fabsf(lead_f32(pc)), fabsf(lead_f32(pm)));
    if (big > 0x1p64f) { pc = scale2(pc, -64); pm = scale2(pm, -64); }
    else if (big < 0x1p-64f) { pc = scale2(pc, 64); pm = scale2(pm, 64); }
  }
  return c;
}

// LU factors with partial pivoting of the tridiagonal T - sigma I (T = (d, e)): u0 holds the
// reciprocals of the pivots, u1, u2 the superdiagonals, lm the multipliers, piv the row swaps;
// a pivot below tiny is raised to tiny (inverse iteration's near-singular shift).  Factor
// entry i sits at [i * s] (several vectors' factors interleaved).
template <typename R>
__device__ __forceinline__ R guard_tiny(R v, R tiny) {
  return (fabs(v) < tiny) ? copysign(tiny, v == R(0.0) ? R(1.0) : v) : v;
}

template <typename R>
__device__ __forceinline__ void tri_shift_factor(const R* __restrict__ d, const R* __restrict__ e, int k, R sigma,
                                                 R tiny, R* __restrict__ u0, R* __restrict__ u1,
                                                 R* __restrict__ u2, R* __restrict__ lm,
                                                 unsigned char* __restrict__ piv, int s) {
  R c0 = d[0] - sigma;                   // running pivot row: (c0, c1, 0) in columns i, i+1, i+2
  R c1 = (k > 1) ? e[0] : R(0.0);
  for (int i = 0; i + 1 < k; ++i) {
    const R sub = e[i];
    const R nd = d[i + 1] - sigma;
    const R ne = (i + 2 < k) ? e[i + 1] : R(0.0);
    if (fabs(c0) >= fabs(sub)) {
      const R rc = R(1.0) / guard_tiny(c0, tiny);
      const R l = sub * rc;
      u0[i * s] = rc; u1[i * s] = c1; u2[i * s] = R(0.0);
      lm[i * s] = l;
      piv[i * s] = 0;
      c0 = dfma(-l, c1, nd);
      c1 = ne;
    } else {
      const R rs = R(1.0) / guard_tiny(sub, tiny);
      const R l = c0 * rs;
      u0[i * s] = rs; u1[i * s] = nd; u2[i * s] = ne;
      lm[i * s] = l;
      piv[i * s] = 1;
      const R t = c1;
      c0 = dfma(-l, nd, t);
      c1 = -l * ne;
    }
  }
  u0[(k - 1) * s] = R(1.0) / guard_tiny(c0, tiny);
}

// y <- (T - sigma I)^{-1} y from the factors of tri_shift_factor.
template <typename R>
__device__ __forceinline__ void tri_shift_apply(int k, const R* __restrict__ u0, const R* __restrict__ u1,
                                                const R* __restrict__ u2, const R* __restrict__ lm,
                                                const unsigned char* __restrict__ piv, int s, R* __restrict__ y) {
  R yc = y[0];
  for (int i = 0; i + 1 < k; ++i) {
    R yn = y[i + 1];
    if (piv[i * s]) { const R t = yc; yc = yn; yn = t; }
    y[i] = yc;
    yc = dfma(-lm[i * s], yc, yn);
  }
  R y1 = yc * u0[(k - 1) * s];           // y[i+1]
  y[k - 1] = y1;
  R y2 = 0.0;                            // y[i+2]
  for (int i = k - 2; i >= 0; --i) {
    const R t = dfma(-u2[i * s], y2, y[i]);
    const R yi = dfma(-u1[i * s], y1, t) * u0[i * s];
    y[i] = yi;
    y2 = y1;
    y1 = yi;
  }
}

// Strided views: element i at p[i * s] (several vectors stored interleaved).
template <typename R>
struct StridedD {
  R* p;
  int s;
  __device__ R& operator[](int i) const { return p[i * s]; }
};
struct StridedB {
  unsigned char* p;
  int s;
  __device__ unsigned char& operator[](int i) const { return p[i * s]; }
};

__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (float)(h & 0xFFFFFF) * 0x1p-23f - 1.0f;  // in [-1, 1), exact
}

// Tridiagonal T y = theta y for the lowest m eigenpairs.  Y (k x m, column t contiguous at
// Y + t*ldy, ldy = k rounded up to odd so that one-thread-per-vector sweeps in shared memory
// do not collide on banks) receives unit eigenvectors, w the eigenvalues (ascending).
template <typename R>
struct TriWork {
  R *d, *e, *u0, *u1, *u2, *lm, *Y, *P;  // u*, lm: m*k each (interleaved); Y: m*ldy; P: 32*32
  int ldy;
  unsigned char* piv;                    // m*k (interleaved)
  R *ds, *e2s;                           // d and e^2 of the tridiagonal scaled by 2^-sexp
  R *lo, *hi;                            // m: bisection brackets (scaled)
  R* xs;                                 // nt: the multisection points of a round
  int* cnt;                              // nt
};

template <typename R>
__device__ void tri_eig_lowest(int k, int m, TriWork<R> W, double* w, R* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // norm bound (max Gershgorin row sum) and the power of two at or above it
  R mx = 0.0;
  for (int i = tid; i < k; i += nt) {
    const R el = (i > 0) ? fabs(W.e[i - 1]) : R(0.0), er = (i + 1 < k) ? fabs(W.e[i]) : R(0.0);
    mx = fmax(mx, fabs(W.d[i]) + el + er);
  }
  const R tnorm = fmax(block_max(mx, red), R(SmallTraits<R>::floor));
  int sexp;
  frexpf(lead_f32(tnorm) * 1.001f, &sexp);   // tnorm <= 2^sexp
  sexp = min(max(sexp, -125), 126);
  // scaled copy (exact) and Gershgorin bounds of the scaled matrix
  R glo = 4.0, ghi = -4.0;
  for (int i = tid; i < k; i += nt) {
    const R di = scale2(W.d[i], -sexp);
    const R el = (i > 0) ? fabs(scale2(W.e[i - 1], -sexp)) : R(0.0);
    const R er = (i + 1 < k) ? fabs(scale2(W.e[i], -sexp)) : R(0.0);
    W.ds[i] = di;
    if (i + 1 < k) W.e2s[i] = er * er;
    glo = fmin(glo, di - el - er);
    ghi = fmax(ghi, di + el + er);
  }
  glo = -block_max(-glo, red);
  ghi = block_max(ghi, red);
  glo -= R(1e-12);
  ghi += R(1e-12);
  // multisection.  Round 0: every thread samples one point of [glo, ghi] (shared by all
  // wanted eigenvalues); eigenvalue t lies where the counts pass t.  Then G lanes per wanted
  // eigenvalue split its bracket into G + 1 parts per round, to the working precision.
  // Invariant: count(lo) <= t < count(hi).
  {
    const R x = dfma(ghi - glo, R((float)(tid + 1) / (float)(nt + 1)), glo);
    W.xs[tid] = x;
    W.cnt[tid] = sturm_count(W.ds, W.e2s, k, x);
  }
  __syncthreads();
  for (int t = tid; t < m; t += nt) {
    int q0 = 0, q1 = nt;   // first sample with count > t (binary search; counts grow with x)
    while (q0 < q1) {
      const int q = (q0 + q1) >> 1;
      if (W.cnt[q] > t) q1 = q; else q0 = q + 1;
    }
    W.lo[t] = (q0 == 0) ? glo : W.xs[q0 - 1];
    W.hi[t] = (q0 == nt) ? ghi : W.xs[q0];
  }
  __syncthreads();
  // rounds 1, 2, ...: G lanes per wanted eigenvalue (G a power of two <= 32, so a warp holds
  // 32 / G of them), the bracket in registers; a ballot over the lanes' counts picks the
  // first point above the eigenvalue, with no barrier
  int G = 32;
  while (G > 1 && G * m > nt) G >>= 1;
  const int lane = tid & 31, seg = lane / G, g = lane % G;
  const int t = (tid >> 5) * (32 / G) + seg;   // this lane's eigenvalue
  const bool has = t < m;
  const unsigned segmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (seg * G));
  const float bits = log2f(lead_f32(ghi - glo) / (float)(nt + 1)) - log2f((float)SmallTraits<R>::eps);
  const int rounds = max(0, (int)ceilf(bits / log2f((float)G + 1.0f)));
  const float frac = (float)(g + 1) / (float)(G + 1);   // this lane's point in the bracket
  R lo = has ? W.lo[t] : R(0.0), hi = has ? W.hi[t] : R(1.0);
  for (int r = 0; r < rounds; ++r) {
    const R x = dfma(hi - lo, R(frac), lo);
    const bool below = has && sturm_count(W.ds, W.e2s, k, x) <= t;
    const unsigned above = ~__ballot_sync(0xffffffffu, below) & segmask;
    const int q = above ? (__ffs(above) - 1 - seg * G) : G;   // points at or below, in order
    const R xl = shfl(x, seg * G + max(q - 1, 0));
    const R xh = shfl(x, seg * G + min(q, G - 1));
    if (q > 0) lo = xl;
    if (q < G) hi = xh;
  }
  __syncthreads();
  if (has && g == 0) {
    W.lo[t] = lo;
    W.hi[t] = hi;
  }
  __syncthreads();
  // inverse iteration, one thread per eigenvector, distinct pseudo-random starts, three solves
  // with the factors of T - lam I at the bisected eigenvalue (each contracts the other
  // eigenvectors' components by ~eps ||T|| / gap, which is not small for the tiny eigenvalues
  // of a graded matrix; closer eigenvalues form the clusters below)
  const R tiny = fmax(R(SmallTraits<R>::eps) * tnorm, R(SmallTraits<R>::tiny_abs));
  for (int t = tid; t < m; t += nt) {
    const R lam = scale2(R(0.5) * (W.lo[t] + W.hi[t]), sexp);
    R* y = W.Y + (size_t)t * W.ldy;
    for (int i = 0; i < k; ++i) y[i] = hash_unit(t + 1, i + 1);
    // the factors of T - lam I serve every solve (interleaved per-vector storage)
    tri_shift_factor(W.d, W.e, k, lam, tiny, W.u0 + t, W.u1 + t, W.u2 + t, W.lm + t, W.piv + t, m);
    bool bad = false;
    for (int it = 0; it < 3 && !bad; ++it) {
      tri_shift_apply(k, W.u0 + t, W.u1 + t, W.u2 + t, W.lm + t, W.piv + t, m, y);
      // rescale by the largest entry: the solve can grow y by up to 1/tiny
      R ymx = 0.0;
      for (int i = 0; i < k; ++i) ymx = fmax(ymx, fabs(y[i]));
      bad = !(ymx > R(0.0)) || !isfinite(ymx);
      if (!bad) {
        const R rmx = R(1.0) / ymx;
        for (int i = 0; i < k; ++i) y[i] *= rmx;
      }
    }
    if (bad) {
      for (int i = 0; i < k; ++i) y[i] = R((i == t % k) ? 1.0 : 0.0);
    } else {
      R n0 = 0.0, n1 = 0.0;
      int i = 0;
      for (; i + 1 < k; i += 2) { n0 = dfma(y[i], y[i], n0); n1 = dfma(y[i + 1], y[i + 1], n1); }
      if (i < k) n0 = dfma(y[i], y[i], n0);
      const R nrm = rsqrt(n0 + n1);
      for (int l = 0; l < k; ++l) y[l] *= nrm;
    }
    w[t] = (double)lam;
  }
  __syncthreads();
  // clusters of close eigenvalues: MGS (warp 0), then diagonalise the projected cluster block
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double ctol = 1e-3 * (double)tnorm;
    int cs = 0;
    for (int t = 1; t <= m; ++t) {
      const bool brk = (t == m) || (w[t] - w[t - 1] > ctol);
      if (!brk) continue;
      const int c = t - cs;
      if (c > 1) {
        for (int a = cs; a < t; ++a) {
          R* ya = W.Y + (size_t)a * W.ldy;
          for (int pass = 0; pass < 2; ++pass) {
            for (int b = cs; b < a; ++b) {
              const R* yb = W.Y + (size_t)b * W.ldy;
              R dt = 0.0;
              for (int i = lane; i < k; i += 32) dt += ya[i] * yb[i];
              dt = wsum(dt);
              for (int i = lane; i < k; i += 32) ya[i] -= dt * yb[i];
              __syncwarp();
            }
          }
          R nn = 0.0;
          for (int i = lane; i < k; i += 32) nn += ya[i] * ya[i];
          nn = rsqrt(fmax(wsum(nn), R(SmallTraits<R>::floor)));
          for (int i = lane; i < k; i += 32) ya[i] *= nn;
          __syncwarp();
        }
        if (c <= 32) {
          // projected block P = Yc^T T Yc (c x c)
          for (int a = 0; a < c; ++a) {
            const R* ya = W.Y + (size_t)(cs + a) * W.ldy;
            for (int b = 0; b <= a; ++b) {
              const R* yb = W.Y + (size_t)(cs + b) * W.ldy;
              R s = 0.0;
              for (int i = lane; i < k; i += 32) {
                R ty = W.d[i] * yb[i];
                if (i > 0) ty += W.e[i - 1] * yb[i - 1];
                if (i + 1 < k) ty += W.e[i] * yb[i + 1];
                s += ya[i] * ty;
              }
              s = wsum(s);
              if (lane == 0) { W.P[a * 32 + b] = s; W.P[b * 32 + a] = s; }
            }
          }
          __syncwarp();
          // cyclic Jacobi on P (lane 0), rotations applied to the cluster vectors by the warp
          for (int sweep = 0; sweep < 30; ++sweep) {
            R off = 0.0;
            if (lane == 0)
              for (int a = 0; a < c; ++a)
                for (int b = 0; b < a; ++b) off += W.P[a * 32 + b] * W.P[a * 32 + b];
            off = shfl(off, 0);
            if (off < R(1e-30) * tnorm * tnorm) break;
            for (int a = 0; a < c; ++a) {
              for (int b = a + 1; b < c; ++b) {
                R cth = 1.0, sth = 0.0;
                if (lane == 0) {
                  const R apq = W.P[a * 32 + b];
                  if (fabs(apq) > R(SmallTraits<R>::floor)) {
                    const R tau = (W.P[b * 32 + b] - W.P[a * 32 + a]) / (R(2.0) * apq);
                    const R tt = copysign(R(1.0), tau) / (fabs(tau) + sqrt(R(1.0) + tau * tau));
                    cth = rsqrt(R(1.0) + tt * tt);
                    sth = tt * cth;
                    for (int r2 = 0; r2 < c; ++r2) {
                      const R pa = W.P[r2 * 32 + a], pb = W.P[r2 * 32 + b];
                      W.P[r2 * 32 + a] = cth * pa - sth * pb;
                      W.P[r2 * 32 + b] = sth * pa + cth * pb;
                    }
                    for (int r2 = 0; r2 < c; ++r2) {
                      const R pa = W.P[a * 32 + r2], pb = W.P[b * 32 + r2];
                      W.P[a * 32 + r2] = cth * pa - sth * pb;
                      W.P[b * 32 + r2] = sth * pa + cth * pb;
                    }
                  }
                }
                cth = shfl(cth, 0);
                sth = shfl(sth, 0);
                if (sth != R(0.0)) {
                  R* ya = W.Y + (size_t)(cs + a) * W.ldy;
                  R* yb = W.Y + (size_t)(cs + b) * W.ldy;
                  for (int i = lane; i < k; i += 32) {
                    const R va = ya[i], vb = yb[i];
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
            R bv = W.P[a * 32 + a];
            for (int b = a + 1; b < c; ++b)
              if (W.P[b * 32 + b] < bv) { bv = W.P[b * 32 + b]; best = b; }
            if (best != a) {
              R* ya = W.Y + (size_t)(cs + a) * W.ldy;
              R* yb = W.Y + (size_t)(cs + best) * W.ldy;
              for (int i = lane; i < k; i += 32) { const R tv = ya[i]; ya[i] = yb[i]; yb[i] = tv; }
              __syncwarp();
              if (lane == 0) {
                const R tv = W.P[a * 32 + a];
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
    const R* y = W.Y + (size_t)t * W.ldy;
    R s = 0.0;
    for (int i = 0; i < k; ++i) {
      R ty = W.d[i] * y[i];
      if (i > 0) ty += W.e[i - 1] * y[i - 1];
      if (i + 1 < k) ty += W.e[i] * y[i + 1];
      s += y[i] * ty;
    }
    w[t] = (double)s;
  }
  __syncthreads();
  // keep ascending order (clusters may reorder neighbours by roundoff): insertion sort by thread 0
  if (tid == 0) {
    for (int a = 1; a < m; ++a) {
      int b = a;
      while (b > 0 && w[b - 1] > w[b]) {
        const double tv = w[b]; w[b] = w[b - 1]; w[b - 1] = tv;
        R* ya = W.Y + (size_t)b * W.ldy;
        R* yb = W.Y + (size_t)(b - 1) * W.ldy;
        for (int i = 0; i < k; ++i) { const R tt = ya[i]; ya[i] = yb[i]; yb[i] = tt; }
        --b;
      }
    }
  }
  __syncthreads();
}

// Z (k x m row-major) = Q Y with Q = H_0 H_1 ... H_{k-3}; Y column t at Y + t*ldy.  One
// half-warp per vector, reflectors in pairs: with a = v_j . y, b = v_{j-1} . y and
// c_j = v_{j-1} . v_j, H_{j-1} H_j y = y - 2 a v_j - 2 (b - 2 a c_j) v_{j-1}, so the two dot
// products of a pair reduce together.  cv: k scalars of scratch for the c_j.
template <typename R, typename ZT>
__device__ void back_transform(int k, int m, const R* V, R* Y, int ldy, ZT* Z, R* cv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 1 + warp; j <= k - 3; j += nw) {
    R s = 0.0;
    for (int i = j + 1 + lane; i < k; i += 32) s = dfma(V[(size_t)(j - 1) * k + i], V[(size_t)j * k + i], s);
    s = wsum(s);
    if (lane == 0) cv[j] = s;
  }
  __syncthreads();
  const int hl = threadIdx.x & 15, hw = threadIdx.x >> 4, nh = blockDim.x >> 4;
  const int tmax = ((m + nh - 1) / nh) * nh;   // uniform trip count: whole warps shuffle
  for (int t0 = 0; t0 < tmax; t0 += nh) {
    const int t = t0 + hw;
    const bool act = t < m;
    R* y = Y + (size_t)(act ? t : 0) * ldy;
    int j = k - 3;
    for (; j >= 1; j -= 2) {
      const R* va = V + (size_t)j * k;         // applied first
      const R* vb = V + (size_t)(j - 1) * k;
      R da = 0.0, db = 0.0;
      if (act)
        for (int i = j + hl; i < k; i += 16) {
          const R yi = y[i];
          da = dfma(va[i], yi, da);
          db = dfma(vb[i], yi, db);
        }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        da = da + shfl_xor(da, o);
        db = db + shfl_xor(db, o);
      }
      const R fa = R(-2.0) * da;
      const R fb = R(-2.0) * dfma(fa, cv[j], db);
      if (act)
        for (int i = j + hl; i < k; i += 16) y[i] = dfma(fb, vb[i], dfma(fa, va[i], y[i]));
      __syncwarp();
    }
    if (j == 0) {
      const R* v = V;
      R dt = 0.0;
      if (act)
        for (int i = 1 + hl; i < k; i += 16) dt = dfma(v[i], y[i], dt);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) dt = dt + shfl_xor(dt, o);
      const R f = R(-2.0) * dt;
      if (act)
        for (int i = 1 + hl; i < k; i += 16) y[i] = dfma(f, v[i], y[i]);
      __syncwarp();
    }
    if (act)
      for (int i = hl; i < k; i += 16) Z[(size_t)i * m + t] = (ZT)y[i];
  }
  __syncthreads();
}

// Workspace layout for a k x k problem with m wanted pairs.
struct SyevLayout {
  size_t a, V, p, vp, d, e, ds, e2s, u0, u1, u2, lm, Y, P, lo, hi, xs, cnt, piv, total;
  int ldy;
  SyevLayout(int k, int m) {
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 127) & ~size_t(127); return r; };
    ldy = k | 1;
    a = take((size_t)k * k * 8); V = take((size_t)k * k * 8); p = take((size_t)k * 8); vp = take((size_t)k * 8);
    d = take((size_t)k * 8); e = take((size_t)k * 8); ds = take((size_t)k * 8); e2s = take((size_t)k * 8);
    u0 = take((size_t)m * k * 8); u1 = take((size_t)m * k * 8); u2 = take((size_t)m * k * 8);
    lm = take((size_t)m * k * 8); Y = take((size_t)m * ldy * 8); P = take(32 * 32 * 8);
    lo = take((size_t)m * 8); hi = take((size_t)m * 8); xs = take(kSmallThreads * 8); cnt = take(kSmallThreads * 4);
    piv = take((size_t)m * k);
    total = o;
  }
};

template <typename R>
__device__ TriWork<R> make_triwork(unsigned char* base, const SyevLayout& L) {
  TriWork<R> W;
  W.d = (R*)(base + L.d); W.e = (R*)(base + L.e);
  W.ds = (R*)(base + L.ds); W.e2s = (R*)(base + L.e2s);
  W.u0 = (R*)(base + L.u0); W.u1 = (R*)(base + L.u1); W.u2 = (R*)(base + L.u2);
  W.lm = (R*)(base + L.lm); W.Y = (R*)(base + L.Y); W.P = (R*)(base + L.P);
  W.ldy = L.ldy;
  W.lo = (R*)(base + L.lo); W.hi = (R*)(base + L.hi); W.xs = (R*)(base + L.xs); W.cnt = (int*)(base + L.cnt);
  W.piv = base + L.piv;
  return W;
}

// Dynamic shared memory for a workspace of `bytes` (0: it stays in global memory).
template <typename K>
static int smem_launch_bytes(K kern, size_t bytes) {
  if (bytes > kSmallSmemBytes) return 0;
  if (::eig::ensure_dyn_smem(kern, bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (int)bytes;
}

// Eigen-decomposition of the symmetric matrix already in L.a (workspace); lowest m.
template <typename R, typename ZT>
__device__ void syev_in_work(unsigned char* base, const SyevLayout& L, int k, int m, double* w, ZT* Z, R* red) {
  R* a = (R*)(base + L.a);
  R* V = (R*)(base + L.V);
  R* p = (R*)(base + L.p);
  R* vp = (R*)(base + L.vp);
  TriWork<R> W = make_triwork<R>(base, L);
  if (k == 1) {
    if (threadIdx.x == 0) { w[0] = (double)a[0]; Z[0] = ZT(1.0); }
    __syncthreads();
    return;
  }
  tridiagonalize(a, k, W.d, W.e, V, p, vp);
  tri_eig_lowest(k, m, W, w, red);
  back_transform(k, m, V, W.Y, W.ldy, Z, p);
}

template <typename R, bool SM>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_syev(const double* A, int k, int m, double* w, double* Z,
                                                              unsigned char* gwork, SyevLayout L, int* info,
                                                              int) {
  __shared__ R red[33];
  extern __shared__ __align__(128) unsigned char s_dyn[];
  unsigned char* work = SM ? s_dyn : gwork;   // compile-time: shared-memory addressing
  R* a = (R*)(work + L.a);
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
    const int r = i / k, c = i % k;
    a[i] = R(0.5 * (A[r * k + c] + A[c * k + r]));
  }
  __syncthreads();
  syev_in_work(work, L, k, m, w, Z, red);
  if (threadIdx.x == 0 && info) *info = SMALL_OK;
}

size_t small_syev_work_bytes(int k, int m) { return SyevLayout(k, m).total; }

// Tridiagonal input (Lanczos T_k of Eq. lanfac): lowest m eigenpairs of (d, e), Z (k x m).
template <typename R, bool SM>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_tri_eig(const double* d, const double* e, int k, int m,
                                                                 double* w, double* Z, unsigned char* gwork,
                                                                 SyevLayout L, int) {
  __shared__ R red[33];
  extern __shared__ __align__(128) unsigned char s_dyn[];
  unsigned char* work = SM ? s_dyn : gwork;   // compile-time: shared-memory addressing
  TriWork<R> W = make_triwork<R>(work, L);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    W.d[i] = R(d[i]);
    W.e[i] = R((i + 1 < k) ? e[i] : 0.0);
  }
  __syncthreads();
  if (k == 1) {
    if (threadIdx.x == 0) { w[0] = (double)W.d[0]; Z[0] = 1.0; }
    return;
  }
  tri_eig_lowest(k, m, W, w, red);
  for (int idx = threadIdx.x; idx < k * m; idx += blockDim.x) {
    const int i = idx / m, t = idx % m;
    Z[idx] = (double)W.Y[(size_t)t * W.ldy + i];
  }
}

eig_status small_tri_eig(const double* d, const double* e, int k, int m, double* w, double* Z, void* work,
                         cudaStream_t st) {
  if (k < 1 || m < 1 || m > k || m > 256) return EIG_EINVAL;
  SyevLayout L(k, m);
  const int sm = smem_launch_bytes(k_small_tri_eig<SmallR, true>, L.total);
  if (sm > 0)
    k_small_tri_eig<SmallR, true><<<1, kSmallThreads, sm, st>>>(d, e, k, m, w, Z, (unsigned char*)work, L, 1);
  else
    k_small_tri_eig<SmallR, false><<<1, kSmallThreads, 0, st>>>(d, e, k, m, w, Z, (unsigned char*)work, L, 0);
  EIG_LAUNCH_CHECK("k_small_tri_eig");
  return EIG_OK;
}

eig_status small_syev(const double* A, int k, int m, double* w, double* Z, void* work, int* info, cudaStream_t st) {
  if (k < 1 || m < 1 || m > k || k > kSmallMax || m > 256) return EIG_EINVAL;
  SyevLayout L(k, m);
  const int sm = smem_launch_bytes(k_small_syev<SmallR, true>, L.total);
  if (sm > 0)
    k_small_syev<SmallR, true><<<1, kSmallThreads, sm, st>>>(A, k, m, w, Z, (unsigned char*)work, L, info, 1);
  else
    k_small_syev<SmallR, false><<<1, kSmallThreads, 0, st>>>(A, k, m, w, Z, (unsigned char*)work, L, info, 0);
  EIG_LAUNCH_CHECK("k_small_syev");
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// Cholesky (lower, in place) of a k x k SPD matrix g, right-looking with one CTA barrier per
// column: column j's scaled entries go to the (unused) strictly upper part while the
// trailing update reads the unscaled column, and a last pass moves them below the diagonal.
// The thread that finishes the next pivot computes its reciprocal root at once.  rd receives
// the reciprocals of L's diagonal.  Breakdown when a pivot <= piv_tol (every thread sees the
// same pivot, so the return value is uniform across the CTA).
// ---------------------------------------------------------------------------------------
template <typename R>
__device__ int cholesky_lower(R* g, int k, double piv_tol, R* rd) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tc = tid & 15, ti = tid >> 4, nr = nt >> 4;
  if (tid == 0) rd[0] = rsqrt(g[0]);
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (!(g[j * k + j] > R(piv_tol))) return SMALL_BREAKDOWN;
    const R rl = rd[j];
    const R rp = rl * rl;
    for (int i = j + 1 + tid; i < k; i += nt) g[j * k + i] = g[i * k + j] * rl;
    // trailing update g[i][l] -= g[i][j] g[l][j] / pivot on the lower triangle: rows
    // j + 1 + ti + nr s, columns j + 1 + tc + 16 u
    for (int i = j + 1 + ti; i < k; i += nr) {
      const R bi = g[i * k + j] * rp;
      int l = j + 1 + tc;
      for (; l + 16 <= i; l += 32) {
        const R a0 = g[i * k + l], a1 = g[i * k + l + 16], c0 = g[l * k + j], c1 = g[(l + 16) * k + j];
        g[i * k + l] = dfma(-bi, c0, a0);
        g[i * k + l + 16] = dfma(-bi, c1, a1);
      }
      if (l <= i) {
        const R r0 = dfma(-bi, g[l * k + j], g[i * k + l]);
        g[i * k + l] = r0;
        if (l == j + 1 && i == j + 1) rd[j + 1] = rsqrt(r0);   // the next pivot is final
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    if (l < i) g[idx] = g[l * k + i];
    else if (l == i) g[idx] = R(1.0) / rd[i];
  }
  __syncthreads();
  return SMALL_OK;
}

// X <- L^{-1} X for lower-triangular L (k x k, row-major, reciprocal diagonal rd) and X
// (k x nc, row-major, leading dimension ldx), by the whole CTA, right-looking: step i
// subtracts the finished row i from the rows below it, and each row is scaled by its
// reciprocal pivot in the step that finishes it.  One barrier per row.
template <typename R>
__device__ void trsm_lower(const R* L, int k, const R* rd, R* X, int ldx, int nc) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tc = tid & 15, ti = tid >> 4, nr = nt >> 4;
  for (int c = tid; c < nc; c += nt) X[c] *= rd[0];
  __syncthreads();
  for (int i = 0; i + 1 < k; ++i) {
    for (int r = i + 1 + ti; r < k; r += nr) {
      const R lri = -L[r * k + i];
      const R s = (r == i + 1) ? rd[r] : R(1.0);
      for (int c = tc; c < nc; c += 16) {
        const R v = dfma(lri, X[i * ldx + c], X[r * ldx + c]);
        X[r * ldx + c] = (r == i + 1) ? v * s : v;
      }
    }
    __syncthreads();
  }
}

// X <- L^{-T} X for the same L, X (k x nc), right-looking backward, two rows per barrier
// (for few columns: every thread finishes the second row for its own columns in registers):
// on entry to a step rows >= i are final and row i - 1 lacks only row i's update; the step
// subtracts rows i and i - 1 from the rows above and finishes row i - 2.  Row i - 1 itself is
// written after the barrier (others read its old value during the step), staged through the
// double-buffered row nxt (2 * nc scalars).
template <typename R>
__device__ void trsm_lower_t(const R* L, int k, const R* rd, R* X, int ldx, int nc, R* nxt) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tc = tid & 15, ti = tid >> 4, nr = nt >> 4;
  for (int c = tid; c < nc; c += nt) X[(k - 1) * ldx + c] *= rd[k - 1];
  __syncthreads();
  int pend = -1;
  int step = 0;
  for (int i = k - 1; i > 0; i -= 2, ++step) {
    R* stage = nxt + (step & 1) * nc;
    if (pend >= 0 && ti == 0)
      for (int c = tc; c < nc; c += 16) X[pend * ldx + c] = nxt[((step - 1) & 1) * nc + c];
    const R l10 = -L[i * k + i - 1], r1 = rd[i - 1];
    for (int c = tc; c < nc; c += 16) {
      const R x0 = X[i * ldx + c];
      const R x1 = dfma(l10, x0, X[(i - 1) * ldx + c]) * r1;
      if (ti == 0) stage[c] = x1;
      for (int r = ti; r < i - 1; r += nr) {
        const R v = dfma(-L[(i - 1) * k + r], x1, dfma(-L[i * k + r], x0, X[r * ldx + c]));
        X[r * ldx + c] = (r == i - 2) ? v * rd[r] : v;
      }
    }
    pend = i - 1;
    __syncthreads();
  }
  if (pend >= 0 && ti == 0)
    for (int c = tc; c < nc; c += 16) X[pend * ldx + c] = nxt[((step - 1) & 1) * nc + c];
  __syncthreads();
}

// Rayleigh-Ritz on (A, G), see small.cuh.
struct RRLayout {
  size_t g, dsc, t, syev, z, nx, total;
  SyevLayout S;
  RRLayout(int k, int nb) : S(k, nb) {
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 127) & ~size_t(127); return r; };
    g = take((size_t)k * k * 8); dsc = take((size_t)k * 2 * 8); t = take((size_t)k * k * 8);
    z = take((size_t)k * nb * 8);
    nx = take((size_t)2 * k * 8);
    syev = take(S.total);
    total = o;
  }
};

template <typename R, bool SM>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_rr(const double* A, const double* G, int k, int nb,
                                                            double piv_tol, int pivoted, double* theta, double* C,
                                                            float* C32, unsigned char* gwork, RRLayout L, int* info,
                                                            int) {
  __shared__ R red[33];
  extern __shared__ __align__(128) unsigned char s_dyn[];
  unsigned char* work = SM ? s_dyn : gwork;   // compile-time: shared-memory addressing
  __shared__ int sel[kSmallMax / 4];
  __shared__ int ksel, pstar;
  __shared__ R dstar;
  const int tid = threadIdx.x, nt = blockDim.x;
  R* g = (R*)(work + L.g);
  R* dsc = (R*)(work + L.dsc);
  R* t = (R*)(work + L.t);
  R* z = (R*)(work + L.z);
  R* nx = (R*)(work + L.nx);
  unsigned char* sw = work + L.syev;
  R* a = (R*)(sw + L.S.a);
  // column scaling to a unit-diagonal Gram
  for (int i = tid; i < k; i += nt) {
    const double gi = G[i * k + i];
    dsc[i] = R((gi > 0.0) ? rsqrt(gi) : 0.0);
  }
  __syncthreads();
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    g[idx] = R(0.5 * (G[i * k + l] + G[l * k + i])) * dsc[i] * dsc[l];
    t[idx] = R(0.5 * (A[i * k + l] + A[l * k + i])) * dsc[i] * dsc[l];
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
        R bd = -1.0;
        for (int i = 0; i < k; ++i)   // taken columns carry -1 on the diagonal
          if (a[i * k + i] > bd) { bd = a[i * k + i]; best = i; }
        pstar = (best >= 0 && bd > R(piv_tol)) ? best : -1;
        dstar = bd;
        if (pstar >= 0) sel[ksel] = pstar;
      }
      __syncthreads();
      if (pstar < 0) break;
      const int p = pstar;
      const R rp = rsqrt(dstar);
      // Schur complement over the columns not yet taken (the taken ones are never read again)
      for (int idx = tid; idx < k * k; idx += nt) {
        const int i = idx / k, l = idx % k;
        if (i != p && l != p) a[idx] -= (a[i * k + p] * rp) * (a[l * k + p] * rp);
      }
      __syncthreads();
      if (tid == 0) {
        for (int i = 0; i < k; ++i) { a[i * k + p] = R(0.0); a[p * k + i] = R(0.0); }
        a[p * k + p] = R(-1.0);   // taken
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
  // the reciprocal diagonal of L lives in dsc's second half (rd), D in dsc
  R* rd = dsc + kk;
  if (cholesky_lower(g, kk, piv_tol, rd) != SMALL_OK) {
    if (tid == 0) *info = SMALL_BREAKDOWN;
    return;
  }
  // W = L^{-1} T (in place in t), then T' = L^{-1} W^T (in a), symmetrised in place
  trsm_lower(g, kk, rd, t, kk, kk);
  for (int idx = tid; idx < kk * kk; idx += nt) a[idx] = t[(idx % kk) * kk + idx / kk];
  __syncthreads();
  trsm_lower(g, kk, rd, a, kk, kk);
  for (int idx = tid; idx < kk * kk; idx += nt) {
    const int i = idx / kk, l = idx % kk;
    if (l < i) {
      const R v = R(0.5) * (a[i * kk + l] + a[l * kk + i]);
      a[i * kk + l] = v;
      a[l * kk + i] = v;
    }
  }
  __syncthreads();
  syev_in_work(sw, L.S, kk, nb, theta, z, red);
  // C = D L^{-T} Z (in place in z)
  trsm_lower_t(g, kk, rd, z, nb, nb, nx);
  if (pivoted) {
    // rows of the taken columns back to their basis positions, zero rows for the others
    for (int idx = tid; idx < k * nb; idx += nt) C[idx] = 0.0;
    __syncthreads();
    for (int idx = tid; idx < kk * nb; idx += nt) C[sel[idx / nb] * nb + idx % nb] = (double)(z[idx] * dsc[idx / nb]);
  } else {
    for (int idx = tid; idx < kk * nb; idx += nt) C[idx] = (double)(z[idx] * dsc[idx / nb]);
  }
  if (C32) {
    __syncthreads();
    for (int idx = tid; idx < k * nb; idx += nt) C32[idx] = (float)C[idx];
  }
  if (tid == 0) *info = SMALL_OK;
}

size_t small_rr_work_bytes(int k, int nb) { return RRLayout(k, nb).total; }

eig_status small_rr(const double* A, const double* G, int k, int nb, double piv_tol, double* theta, double* C,
                    float* C32, void* work, int* info, cudaStream_t st, int pivoted) {
  if (k < 1 || nb < 1 || nb > k || k > kSmallMax * 4) return EIG_EINVAL;
  if (pivoted && k > kSmallMax / 4) return EIG_EINVAL;
  RRLayout L(k, nb);
  const int sm = smem_launch_bytes(k_small_rr<SmallR, true>, L.total);
  if (sm > 0)
    k_small_rr<SmallR, true><<<1, kSmallThreads, sm, st>>>(A, G, k, nb, piv_tol, pivoted, theta, C, C32,
                                                            (unsigned char*)work, L, info, 1);
  else
    k_small_rr<SmallR, false><<<1, kSmallThreads, 0, st>>>(A, G, k, nb, piv_tol, pivoted, theta, C, C32,
                                                             (unsigned char*)work, L, info, 0);
  EIG_LAUNCH_CHECK("k_small_rr");
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// CholQR factor: G = R^T R, R upper, Rinv = R^{-1}
// ---------------------------------------------------------------------------------------
template <typename S, bool SM>
__global__ void __launch_bounds__(kSmallThreads, 1) k_small_chol_inv(const double* G, int k, double piv_tol, double* R,
                                                                     double* Rinv, float* Rinv32, double* gwork,
                                                                     int* info, int) {
  __shared__ S red[33];
  extern __shared__ __align__(128) unsigned char s_dyn[];
  S* g = SM ? reinterpret_cast<S*>(s_dyn) : reinterpret_cast<S*>(gwork);  // k*k: the factor L
  S* li = g + (size_t)k * k;                                                   // k*k: L^{-1}
  S* rd = li + (size_t)k * k;                                                  // k
  const int tid = threadIdx.x, nt = blockDim.x;
  S md = 0.0;
  for (int i = tid; i < k; i += nt) md = fmax(md, S(G[i * k + i]));
  md = block_max(md, red);
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    g[idx] = S(0.5 * (G[i * k + l] + G[l * k + i]));
    li[idx] = S((i == l) ? 1.0 : 0.0);
  }
  __syncthreads();
  if (cholesky_lower(g, k, piv_tol * (double)md, rd) != SMALL_OK) {
    if (tid == 0) *info = SMALL_BREAKDOWN;
    return;
  }
  // L^{-1}: R = L^T, Rinv = L^{-T} = (L^{-1})^T
  trsm_lower(g, k, rd, li, k, k);
  for (int idx = tid; idx < k * k; idx += nt) {
    const int i = idx / k, l = idx % k;
    R[idx] = (l >= i) ? (double)g[l * k + i] : 0.0;
    const double ri = (l >= i) ? (double)li[l * k + i] : 0.0;
    Rinv[idx] = ri;
    if (Rinv32) Rinv32[idx] = (float)ri;
  }
  if (tid == 0) *info = SMALL_OK;
}

eig_status small_chol_inv(const double* G, int k, double piv_tol, double* R, double* Rinv, float* Rinv32, void* work,
                          int* info, cudaStream_t st) {
  if (k < 1 || k > kSmallMax * 4) return EIG_EINVAL;
  const int sm = smem_launch_bytes(k_small_chol_inv<SmallR, true>, small_chol_inv_work_bytes(k));
  if (sm > 0)
    k_small_chol_inv<SmallR, true><<<1, kSmallThreads, sm, st>>>(G, k, piv_tol, R, Rinv, Rinv32, (double*)work, info, 1);
  else
    k_small_chol_inv<SmallR, false><<<1, kSmallThreads, 0, st>>>(G, k, piv_tol, R, Rinv, Rinv32, (double*)work, info, 0);
  EIG_LAUNCH_CHECK("k_small_chol_inv");
  return EIG_OK;
}

size_t small_chol_inv_work_bytes(int k) { return ((size_t)2 * k * k + k) * 8; }

}  // namespace eig
