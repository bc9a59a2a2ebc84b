// Tall-skinny dense kernels: Gram products (Eq. rreig's S^T S and S^T H S; Eq. bgs's V^T W),
// block-times-small-matrix products (Eqs. xupd, pupd; CholQR's X R^{-1}), the fused LOBPCG
// update, and deterministic reductions.  All are HBM-bound passes over n x nb blocks.
#include "common.cuh"
#include "dense.cuh"
#include "vec.cuh"

namespace eig {

// ---------------------------------------------------------------------------------------
// double-float accumulation in FP32 (Knuth TwoSum + Fast2Sum)
// ---------------------------------------------------------------------------------------
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void df_add(DF& a, float x) {
  const float s = a.hi + x;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (x - bb);
  const float e = err + a.lo;
  const float h = s + e;
  a.lo = e - (h - s);
  a.hi = h;
}

template <typename T> struct Acc;  // chunk accumulator type per vector type
template <> struct Acc<float> { typedef DF type; };
template <> struct Acc<double> { typedef double type; };

__device__ __forceinline__ void acc_zero(DF& a) { a.hi = 0.f; a.lo = 0.f; }
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void acc_add(DF& a, float x) { df_add(a, x); }
__device__ __forceinline__ void acc_add(double& a, double x) { a += x; }
__device__ __forceinline__ double acc_get(const DF& a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double acc_get(const double& a) { return a; }

constexpr int kGramThreads = 256;
constexpr int kGramRows = 32;

struct PairList {
  int a[kMaxPairs], b[kMaxPairs];
  int n;
};

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills the 16 bytes with zeros.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One row of a thread's TM x TM tile: its TM values of each block from shared memory (16-byte
// loads where the tile is 16 bytes wide: rows are nb % TM == 0 elements, tiles TM-aligned, stages
// 16-byte aligned), and the TM x TM products into the chunk sums, FP32 pairs by the FP32x2 FMA
// (each element a single fused, round-to-nearest operation, as with fma).
template <typename T, int TM> struct GramRow {
  __device__ __forceinline__ static void load(const T* p, T* v) {
#pragma unroll
    for (int i = 0; i < TM; ++i) v[i] = p[i];
  }
  __device__ __forceinline__ static void fma(const T* a, const T* b, T (*c)[TM]) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) c[i][j] = ::fma(a[i], b[j], c[i][j]);
  }
};
template <> struct GramRow<float, 4> {
  __device__ __forceinline__ static void load(const float* p, float* v) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  __device__ __forceinline__ static void fma(const float* a, const float* b, float (*c)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 ai = make_float2(a[i], a[i]);
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        const float2 r = __ffma2_rn(ai, make_float2(b[j], b[j + 1]), make_float2(c[i][j], c[i][j + 1]));
        c[i][j] = r.x;
        c[i][j + 1] = r.y;
      }
    }
  }
};
template <> struct GramRow<double, 4> {
  __device__ __forceinline__ static void load(const double* p, double* v) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
  __device__ __forceinline__ static void fma(const double* a, const double* b, double (*c)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) c[i][j] = ::fma(a[i], b[j], c[i][j]);
  }
};

// Thread t owns tiles t, t+256, ... of the (pair, ti, tj) grid of TM x TM tiles.  PIPE: the
// chunks are staged by 16-byte cp.async copies into two shared-memory stages, the next chunk's
// copies in flight while the current one is multiplied (rows of nb values must be a multiple of
// 16 bytes and every block 16-byte aligned); the products and their order are the same either way.
template <typename T, int TM, int MAXT, bool PIPE>
__global__ void __launch_bounds__(kGramThreads)
k_gram(BlockList blocks, PairList pairs, int nb, int64_t n, int64_t rows_per_cta, double* part) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm_base = reinterpret_cast<T*>(sm_raw);  // [stages][nblocks][kGramRows][nb]
  const size_t stage_elems = (size_t)blocks.n * kGramRows * nb;
  typedef typename Acc<T>::type A;
  const int tpp = (nb / TM) * (nb / TM);
  const int ntiles = pairs.n * tpp;     // <= MAXT * kGramThreads
  A acc[MAXT][TM][TM];
  T cacc[MAXT][TM][TM];
#pragma unroll
  for (int s = 0; s < MAXT; ++s)
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) { acc_zero(acc[s][i][j]); cacc[s][i][j] = T(0); }
  const int64_t r0 = blockIdx.x * rows_per_cta;
  const int64_t r1 = min64(n, r0 + rows_per_cta);
  constexpr int EPC = 16 / sizeof(T);                // elements per 16-byte copy
  auto issue = [&](int64_t rc, T* stage) {           // copies of the chunk at row rc
    const int rows = (int)min64(kGramRows, r1 - rc);
    const int per_block = kGramRows * nb / EPC;
    for (int i = threadIdx.x; i < blocks.n * per_block; i += blockDim.x) {
      const int b = i / per_block, e = (i % per_block) * EPC;
      const T* src = static_cast<const T*>(blocks.p[b]) + rc * nb + e;
      const bool in = e < rows * nb;
      cp_async16(stage + (size_t)b * kGramRows * nb + e, in ? (const void*)src : blocks.p[b], in ? 16 : 0);
    }
    cp_async_commit();
  };
  if (PIPE && r0 < r1) issue(r0, sm_base);
  int stage_i = 0;
  for (int64_t rc = r0; rc < r1; rc += kGramRows) {
    const int rows = (int)min64(kGramRows, r1 - rc);
    T* sm = sm_base + (PIPE ? (size_t)stage_i * stage_elems : 0);
    if (PIPE) {
      // the other stage was last read in the previous iteration: every thread is past it
      __syncthreads();
      if (rc + kGramRows < r1) {
        issue(rc + kGramRows, sm_base + (size_t)(stage_i ^ 1) * stage_elems);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      stage_i ^= 1;
    } else {
      __syncthreads();
      for (int b = 0; b < blocks.n; ++b) {
        const T* src = static_cast<const T*>(blocks.p[b]) + rc * nb;
        T* dst = sm + (size_t)b * kGramRows * nb;
        for (int i = threadIdx.x; i < kGramRows * nb; i += blockDim.x) dst[i] = (i < rows * nb) ? src[i] : T(0);
      }
      __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < MAXT; ++s) {
      const int tile = threadIdx.x + s * kGramThreads;
      if (tile < ntiles) {
        const int q = tile / tpp, rem = tile % tpp;
        const int ti = (rem / (nb / TM)) * TM, tj = (rem % (nb / TM)) * TM;
        const T* Ab = sm + (size_t)pairs.a[q] * kGramRows * nb;
        const T* Bb = sm + (size_t)pairs.b[q] * kGramRows * nb;
        for (int r = 0; r < kGramRows; ++r) {
          T av[TM], bv[TM];
          GramRow<T, TM>::load(Ab + r * nb + ti, av);
          GramRow<T, TM>::load(Bb + r * nb + tj, bv);
          GramRow<T, TM>::fma(av, bv, cacc[s]);
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) { acc_add(acc[s][i][j], cacc[s][i][j]); cacc[s][i][j] = T(0); }
      }
    }
  }
  double* out = part + (size_t)blockIdx.x * pairs.n * nb * nb;
#pragma unroll
  for (int s = 0; s < MAXT; ++s) {
    const int tile = threadIdx.x + s * kGramThreads;
    if (tile < ntiles) {
      const int q = tile / tpp, rem = tile % tpp;
      const int ti = (rem / (nb / TM)) * TM, tj = (rem % (nb / TM)) * TM;
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) out[(size_t)q * nb * nb + (ti + i) * nb + tj + j] = acc_get(acc[s][i][j]);
    }
  }
}

// out[j] = sum over parts in fixed order: one warp per output, lane l adds parts l, l+32, ...,
// then a fixed xor tree (bitwise reproducible, and the loads of a warp are independent).
__global__ void k_reduce_partials(const double* __restrict__ part, int nparts, int m, double* __restrict__ out) {
  const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= m) return;
  double s = 0.0;
  for (int b = lane; b < nparts; b += 32) s += part[(size_t)b * m + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[j] = s;
}

// Two CTAs per SM.  The grid also fixes how the rows are grouped into partial sums, and so the
// rounding of every Gram: the hybrid's RMM-DIIS iteration count is sensitive to it (measured at
// n = 2M: 7 iterations with this grouping, 21 with four CTAs per SM).
static int gram_grid(int64_t n, int64_t* rows_per_cta, int max_parts) {
  int g = num_sms() * 2;
  if (max_parts > 0 && g > max_parts) g = max_parts;
  int64_t rpc = (n + g - 1) / g;
  rpc = ((rpc + kGramRows - 1) / kGramRows) * kGramRows;
  if (rpc < kGramRows) rpc = kGramRows;
  g = (int)((n + rpc - 1) / rpc);
  *rows_per_cta = rpc;
  return g;
}

size_t gram_scratch_bytes(int npairs, int nb) { return (size_t)num_sms() * 2 * npairs * nb * nb * 8 + 256; }

eig_status reduce_partials(const double* part, int nparts, int m, double* out, cudaStream_t st) {
  k_reduce_partials<<<(unsigned)(((int64_t)m * 32 + 255) / 256), 256, 0, st>>>(part, nparts, m, out);
  EIG_LAUNCH_CHECK("k_reduce_partials");
  return EIG_OK;
}

template <typename T, int TM>
static eig_status gram_launch(const BlockList& blocks, const PairList& pl, int nb, int64_t n, double* G, void* part,
                              cudaStream_t st, int max_parts) {
  int64_t rpc;
  const int g = gram_grid(n, &rpc, max_parts);
  bool pipe = (nb * sizeof(T)) % 16 == 0;
  for (int b = 0; b < blocks.n; ++b) pipe = pipe && (reinterpret_cast<uintptr_t>(blocks.p[b]) % 16 == 0);
  pipe = pipe && 2 * (size_t)blocks.n * kGramRows * nb * sizeof(T) <= 200 * 1024;
  const size_t sm = (size_t)(pipe ? 2 : 1) * blocks.n * kGramRows * nb * sizeof(T);
  const int ntiles = pl.n * (nb / TM) * (nb / TM);
  auto kern = pipe ? ((ntiles <= kGramThreads) ? k_gram<T, TM, 1, true>
                      : (ntiles <= 2 * kGramThreads ? k_gram<T, TM, 2, true> : k_gram<T, TM, 4, true>))
                   : ((ntiles <= kGramThreads) ? k_gram<T, TM, 1, false>
                      : (ntiles <= 2 * kGramThreads ? k_gram<T, TM, 2, false> : k_gram<T, TM, 4, false>));
  if (sm > 48 * 1024) EIG_CUDA_TRY(::eig::ensure_dyn_smem(kern, (int)sm));
  kern<<<g, kGramThreads, sm, st>>>(blocks, pl, nb, n, rpc, static_cast<double*>(part));
  EIG_LAUNCH_CHECK("k_gram");
  return reduce_partials(static_cast<double*>(part), g, pl.n * nb * nb, G, st);
}

eig_status gram_multi(const BlockList& blocks, const int* pa, const int* pb, int npairs, int nb, int64_t n,
                      eig_dtype vt, double* G, void* part, cudaStream_t st, int max_parts) {
  if (npairs < 1 || npairs > kMaxPairs || nb < 1 || nb > 64 || n < 1 || blocks.n < 1 || blocks.n > 16) return EIG_EINVAL;
  PairList pl;
  pl.n = npairs;
  for (int q = 0; q < npairs; ++q) {
    if (pa[q] < 0 || pa[q] >= blocks.n || pb[q] < 0 || pb[q] >= blocks.n) return EIG_EINVAL;
    pl.a[q] = pa[q];
    pl.b[q] = pb[q];
  }
  const int TM = (nb % 4 == 0) ? 4 : ((nb % 2 == 0) ? 2 : 1);
  if ((size_t)npairs * (nb / TM) * (nb / TM) > 4 * kGramThreads) return EIG_EUNSUPPORTED;
  if (vt == EIG_F32) {
    if (TM == 4) return gram_launch<float, 4>(blocks, pl, nb, n, G, part, st, max_parts);
    if (TM == 2) return gram_launch<float, 2>(blocks, pl, nb, n, G, part, st, max_parts);
    return gram_launch<float, 1>(blocks, pl, nb, n, G, part, st, max_parts);
  }
  if (vt == EIG_F64) {
    if (TM == 4) return gram_launch<double, 4>(blocks, pl, nb, n, G, part, st, max_parts);
    if (TM == 2) return gram_launch<double, 2>(blocks, pl, nb, n, G, part, st, max_parts);
    return gram_launch<double, 1>(blocks, pl, nb, n, G, part, st, max_parts);
  }
  return EIG_EINVAL;
}

// ---------------------------------------------------------------------------------------
// Out = sum_s In_s M_s (+ beta Out): thread per (row, output column)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void k_block_apply(BlockList in, int nb, const double* __restrict__ M, int m, T* __restrict__ Out,
                              double beta, int64_t n) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sM = reinterpret_cast<T*>(sm_raw);  // K x m
  const int K = in.n * nb;
  for (int i = threadIdx.x; i < K * m; i += blockDim.x) sM[i] = (T)M[i];
  __syncthreads();
  const int64_t total = n * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / m;
    const int j = (int)(idx % m);
    T acc = T(0);
    for (int s = 0; s < in.n; ++s) {
      const T* row = static_cast<const T*>(in.p[s]) + r * nb;
      const T* Ms = sM + (size_t)s * nb * m + j;
      for (int k = 0; k < nb; ++k) acc = fma(__ldg(row + k), Ms[(size_t)k * m], acc);
    }
    if (beta != 0.0) acc = fma((T)beta, Out[idx], acc);
    Out[idx] = acc;
  }
}

eig_status block_apply(const BlockList& in, int nb, const double* M, int m, void* Out, double beta, int64_t n,
                       eig_dtype vt, cudaStream_t st) {
  if (in.n < 1 || in.n > kMaxBlocks || nb < 1 || m < 1 || m > 64 || in.n * nb > 1024) return EIG_EINVAL;
  const int grid = num_sms() * 8;
  if (vt == EIG_F32) {
    const size_t sm = (size_t)in.n * nb * m * 4;
    if (sm > 48 * 1024) EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_block_apply<float>, (int)sm));
    k_block_apply<float><<<grid, 256, sm, st>>>(in, nb, M, m, static_cast<float*>(Out), beta, n);
  } else if (vt == EIG_F64) {
    const size_t sm = (size_t)in.n * nb * m * 8;
    if (sm > 48 * 1024) EIG_CUDA_TRY(::eig::ensure_dyn_smem(k_block_apply<double>, (int)sm));
    k_block_apply<double><<<grid, 256, sm, st>>>(in, nb, M, m, static_cast<double*>(Out), beta, n);
  } else {
    return EIG_EINVAL;
  }
  EIG_LAUNCH_CHECK("k_block_apply");
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// conversions, column sums of squares
// ---------------------------------------------------------------------------------------
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ s, B* __restrict__ d, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = (B)s[i];
}

eig_status convert(const void* src, eig_dtype st_, void* dst, eig_dtype dt_, int64_t count, cudaStream_t st) {
  const int grid = num_sms() * 8;
  if (st_ == EIG_F64 && dt_ == EIG_F32) k_convert<double, float><<<grid, 256, 0, st>>>((const double*)src, (float*)dst, count);
  else if (st_ == EIG_F32 && dt_ == EIG_F64) k_convert<float, double><<<grid, 256, 0, st>>>((const float*)src, (double*)dst, count);
  else if (st_ == EIG_F64 && dt_ == EIG_F64) k_convert<double, double><<<grid, 256, 0, st>>>((const double*)src, (double*)dst, count);
  else if (st_ == EIG_F32 && dt_ == EIG_F32) k_convert<float, float><<<grid, 256, 0, st>>>((const float*)src, (float*)dst, count);
  else return EIG_EINVAL;
  EIG_LAUNCH_CHECK("k_convert");
  return EIG_OK;
}

template <typename T>
__global__ void k_col_sumsq(const T* __restrict__ X, int k, int64_t n, double* __restrict__ part) {
  // thread handles column j = tid % k of rows tid/k, tid/k + stride...
  __shared__ double red[1024];
  const int rows_per_pass = blockDim.x / k;
  const int j = threadIdx.x % k, rr = threadIdx.x / k;
  double s = 0.0;
  if (rr < rows_per_pass) {
    for (int64_t r = blockIdx.x * (int64_t)rows_per_pass + rr; r < n; r += (int64_t)gridDim.x * rows_per_pass) {
      const double v = (double)X[r * k + j];
      s += v * v;
    }
  }
  red[threadIdx.x] = (rr < rows_per_pass) ? s : 0.0;
  __syncthreads();
  if (threadIdx.x < k) {
    double t = 0.0;
    for (int q = 0; q < rows_per_pass; ++q) t += red[q * k + threadIdx.x];
    part[(size_t)blockIdx.x * k + threadIdx.x] = t;
  }
}

size_t colsum_scratch_bytes(int k) { return (size_t)num_sms() * 4 * k * 8 + 256; }

eig_status col_sumsq(const void* X, int k, int64_t n, eig_dtype vt, double* out, void* part, cudaStream_t st) {
  if (k < 1 || k > 256) return EIG_EINVAL;
  const int grid = num_sms() * 4;
  const int threads = (256 / k) * k;
  if (vt == EIG_F32) k_col_sumsq<float><<<grid, threads, 0, st>>>((const float*)X, k, n, (double*)part);
  else if (vt == EIG_F64) k_col_sumsq<double><<<grid, threads, 0, st>>>((const double*)X, k, n, (double*)part);
  else return EIG_EINVAL;
  EIG_LAUNCH_CHECK("k_col_sumsq");
  return reduce_partials((const double*)part, grid, k, out, st);
}

// ---------------------------------------------------------------------------------------
// fused LOBPCG update: thread per (row, column j); a CTA covers rows_per_cta rows
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double jacobi_den(double d, double th, double floor) {
  double den = d - th;
  const double mag = fmax(fabs(den), floor);
  return den < 0.0 ? -mag : mag;
}

// Jacobi denominator H_ii - theta, magnitude floored; FP32 is enough for a preconditioner.
__device__ __forceinline__ float jacobi_den_f(double d, double th, float floor) {
  const float den = (float)d - (float)th;
  const float mag = fmaxf(fabsf(den), floor);
  return den < 0.0f ? -mag : mag;
}

// Thread per (row, CPT adjacent columns), three CTAs per SM (80 registers); rows are read with
// 16-byte moves, the Rayleigh-Ritz coefficients come from shared memory as CPT-wide vectors.  In
// place: the lanes of a row (one warp) have read all their inputs before any of them writes
// (__syncwarp).
template <typename T, int NB>
__global__ void __launch_bounds__(256, 3)
k_lobpcg_update(T* __restrict__ X, T* __restrict__ W, T* __restrict__ P, T* __restrict__ HX,
                const T* __restrict__ HW, T* __restrict__ HP, const double* __restrict__ C, int k,
                const double* __restrict__ theta, const double* __restrict__ diagH, double floor, int precond,
                int64_t n, double* __restrict__ part) {
  constexpr int CPT = (NB * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : NB;
  constexpr int LPR = NB / CPT;           // lanes per row
  constexpr int RPP = 256 / LPR;          // rows per pass
  __shared__ __align__(16) T sC[3 * NB * NB];
  __shared__ double red[256 * CPT];
  for (int i = threadIdx.x; i < k * NB; i += blockDim.x) sC[i] = (T)C[i];
  __syncthreads();
  const int j0 = (threadIdx.x % LPR) * CPT, rr = threadIdx.x / LPR;
  double th[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) th[c] = theta[j0 + c];
  double rsq[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) rsq[c] = 0.0;
  float rh[CPT], rl[CPT];  // FP32 rows: double-float sums of squares
#pragma unroll
  for (int c = 0; c < CPT; ++c) rh[c] = rl[c] = 0.0f;
  // acc += A_row * Cblk[:, j0..j0+CPT) and hacc += HA_row * Cblk
  auto gemv2 = [&](const T* A, const T* HA, int cb, Vec<T, CPT>& acc, Vec<T, CPT>& hacc) {
#pragma unroll
    for (int l0 = 0; l0 < NB; l0 += CPT) {
      const Vec<T, CPT> a = VecIO<T, CPT>::ld(A + l0);
      const Vec<T, CPT> ha = VecIO<T, CPT>::ld(HA + l0);
#pragma unroll
      for (int v = 0; v < CPT; ++v) {
        const Vec<T, CPT> cv = VecIO<T, CPT>::ld(sC + (cb + l0 + v) * NB + j0);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          acc.v[c] = fma(a.v[v], cv.v[c], acc.v[c]);
          hacc.v[c] = fma(ha.v[v], cv.v[c], hacc.v[c]);
        }
      }
    }
  };
  // the loop bound is uniform across the CTA so that __syncwarp sees every lane
  for (int64_t base = blockIdx.x * (int64_t)RPP; base < n; base += (int64_t)gridDim.x * RPP) {
    const int64_t r = base + rr;
    const bool valid = r < n;
    Vec<T, CPT> xn, hxn, pn, hpn, wn;
    xn.zero(); hxn.zero(); pn.zero(); hpn.zero(); wn.zero();
    if (valid) {
      if (k == NB) {
        xn = VecIO<T, CPT>::ld(X + r * NB + j0);
        hxn = VecIO<T, CPT>::ld(HX + r * NB + j0);
      } else {
        gemv2(X + r * NB, HX + r * NB, 0, xn, hxn);
        gemv2(W + r * NB, HW + r * NB, NB, pn, hpn);
        if (k == 3 * NB) gemv2(P + r * NB, HP + r * NB, 2 * NB, pn, hpn);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          xn.v[c] += pn.v[c];
          hxn.v[c] += hpn.v[c];
        }
      }
      const double d = diagH[r];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const T res = hxn.v[c] - (T)th[c] * xn.v[c];
        if (sizeof(T) == 4) {
          // exact FP32 square summed in double-float
          const float f = (float)res, p = f * f, pe = fmaf(f, f, -p);
          const float s = rh[c] + p, bb = s - rh[c];
          rl[c] += ((rh[c] - (s - bb)) + (p - bb)) + pe;
          rh[c] = s;
          wn.v[c] = precond == 1 ? (T)(f / jacobi_den_f(d, th[c], (float)floor)) : res;
        } else {
          rsq[c] = fma((double)res, (double)res, rsq[c]);
          wn.v[c] = precond == 1 ? (T)((double)res / jacobi_den(d, th[c], floor)) : res;
        }
      }
    }
    __syncwarp();
    if (valid) {
      if (k != NB) {
        VecIO<T, CPT>::st(X + r * NB + j0, xn);
        VecIO<T, CPT>::st(HX + r * NB + j0, hxn);
        VecIO<T, CPT>::st(P + r * NB + j0, pn);
        VecIO<T, CPT>::st(HP + r * NB + j0, hpn);
      }
      VecIO<T, CPT>::st(W + r * NB + j0, wn);
    }
  }
#pragma unroll
  for (int c = 0; c < CPT; ++c) red[threadIdx.x * CPT + c] = rsq[c] + (double)rh[c] + (double)rl[c];
  __syncthreads();
  for (int j = threadIdx.x; j < NB; j += blockDim.x) {
    const int g = j / CPT, c = j % CPT;
    double t = 0.0;
    for (int q = 0; q < RPP; ++q) t += red[(q * LPR + g) * CPT + c];
    part[(size_t)blockIdx.x * NB + j] = t;
  }
}

int update_grid(int64_t n) {
  int64_t g = (n + 63) / 64;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

eig_status lobpcg_update(void* X, void* W, void* P, void* HX, void* HW, void* HP, const double* C, int k, int nb,
                         const double* theta, const double* diagH, double floor, int precond, int64_t n,
                         eig_dtype vt, double* part, int nparts_max, int* nparts_out, cudaStream_t st) {
  if (nb < 1 || nb > 32 || 32 % nb != 0 || (k != nb && k != 2 * nb && k != 3 * nb)) return EIG_EINVAL;
  const int grid = update_grid(n);
  if (grid > nparts_max) return EIG_EINVAL;
#define EIG_UPD(T, NBV)                                                                                    \
  k_lobpcg_update<T, NBV><<<grid, 256, 0, st>>>((T*)X, (T*)W, (T*)P, (T*)HX, (const T*)HW, (T*)HP, C, k, theta, \
                                                diagH, floor, precond, n, part)
#define EIG_UPD_NB(T)                  \
  switch (nb) {                        \
    case 1: EIG_UPD(T, 1); break;      \
    case 2: EIG_UPD(T, 2); break;      \
    case 4: EIG_UPD(T, 4); break;      \
    case 8: EIG_UPD(T, 8); break;      \
    case 16: EIG_UPD(T, 16); break;    \
    default: EIG_UPD(T, 32); break;    \
  }
  if (vt == EIG_F32) {
    EIG_UPD_NB(float)
  } else if (vt == EIG_F64) {
    EIG_UPD_NB(double)
  } else {
    return EIG_EINVAL;
  }
#undef EIG_UPD_NB
#undef EIG_UPD
  EIG_LAUNCH_CHECK("k_lobpcg_update");
  *nparts_out = grid;
  return EIG_OK;
}

template <typename T>
__global__ void k_jacobi(T* __restrict__ R, const double* __restrict__ theta, const double* __restrict__ diagH,
                         double floor, int nb, int64_t n) {
  const int64_t total = n * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nb;
    const int j = (int)(i % nb);
    R[i] = (T)((double)R[i] / jacobi_den(diagH[r], theta[j], floor));
  }
}

eig_status jacobi_block(void* R, const double* theta, const double* diagH, double floor, int nb, int64_t n,
                        eig_dtype vt, cudaStream_t st) {
  const int grid = num_sms() * 8;
  if (vt == EIG_F32) k_jacobi<float><<<grid, 256, 0, st>>>((float*)R, theta, diagH, floor, nb, n);
  else if (vt == EIG_F64) k_jacobi<double><<<grid, 256, 0, st>>>((double*)R, theta, diagH, floor, nb, n);
  else return EIG_EINVAL;
  EIG_LAUNCH_CHECK("k_jacobi");
  return EIG_OK;
}

}  // namespace eig
