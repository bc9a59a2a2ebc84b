// Mirrored-tile SpMM: Y = H X with H = U + U_strict^T given by its stored upper triangle U
// (Sec. 1; Eqs. upd1-upd2; half storage of Sec. 3.1 is the input format), GB300 layout.
//
// Why mirror.  In the half-stored kernels every stored h_ij feeds two products: a gather
// y_i += h_ij x_j and a scatter z_j += h_ij x_i.  On sm_103a both run out of shared memory and
// the scatter costs a read-modify-write of an nb-wide row per nonzero plus a reduction of the
// warps' private partials; measured, that kernel is bound by the shared-memory pipe at ~4
// wavefronts per nonzero while HBM idles.  Here the plan expands U once, on the device, into
// both triangles, so the kernel only gathers: ~0.6 wavefronts per nonzero of H, at the price of
// storing the strict lower triangle a second time (1-byte columns keep it to ~5 B per entry).
//
// Layout.  Row blocks of 256 rows (one CTA each), column blocks of 64 (a tile); inside a tile
// the rows form 32 groups of 8.  A group's entries are stored as "quads": quad q of group g holds
// step 4q..4q+3 of each of the group's 8 rows, as 32 (uint8 column in tile, value) slots ordered
// [row][step]; rows shorter than the group's longest are padded with column 0xFF.  A chunk is
// a run of consecutive groups of one tile (at most cap quads), with a 32-byte table of each
// group's quad count; chunks of a row block are stored back to back, so a CTA streams them with
// 1-D bulk copies (TMA) through a two-stage mbarrier pipeline.
//
// Kernel.  Lane (slot, q): the slot picks one (row, step-phase) of the warp's current group, q a
// 16-byte slice of the nb-wide X row.  Each row's y stays in registers for the whole row block
// and is written once.  X_J is staged per chunk and replicated across the 128-byte bank lines so
// that the lanes of one shared-memory wavefront always read different copies: the gathers are
// free of bank conflicts whatever the column indices.  The summation order is fixed (chunks,
// quads, steps, then a fixed shuffle tree), so Y is bitwise reproducible.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "spmm.cuh"
#include "tma.cuh"
#include "vec.cuh"

namespace eig {

namespace {

constexpr int kMR = 256;                 // rows per row block
constexpr int kMC = 64;                  // columns per tile
constexpr int kMG = 8;                   // rows per group
constexpr int kMGroups = kMR / kMG;      // groups per tile
constexpr unsigned kPadCol = 0xFFu;

// ---------------------------------------------------------------------------------------
// Plan: both triangles as a CSR, built from U without sorting and without atomics on values
// ---------------------------------------------------------------------------------------

// Entries of row r with columns in [lo, hi) (rows are sorted): [*a, *b).
__device__ __forceinline__ void row_segment(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                            int64_t r, int64_t lo, int64_t hi, int64_t* a, int64_t* b) {
  int64_t L = rowptr[r], H = rowptr[r + 1];
  const int64_t end = H;
  while (L < H) {
    const int64_t m = (L + H) >> 1;
    if (col[m] < lo) L = m + 1; else H = m;
  }
  *a = L;
  H = end;
  while (L < H) {
    const int64_t m = (L + H) >> 1;
    if (col[m] < hi) L = m + 1; else H = m;
  }
  *b = L;
}

// Column-major bitmap of the strictly-upper entries of upper tile t (256 rows x 64 columns):
// bits[j * 8 + w] bit b <=> entry (row 32 w + b, column j).  One thread per row.
__device__ void tile_bits(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          int64_t r0, int64_t cb0, unsigned* bits, int64_t* a, int64_t* b) {
  const int tid = threadIdx.x;
  for (int i = tid; i < kMC * (kMR / 32); i += blockDim.x) bits[i] = 0u;
  __syncthreads();
  const int64_t r = r0 + tid;
  *a = *b = 0;
  if (r < n) {
    row_segment(rowptr, col, r, cb0, cb0 + kMC, a, b);
    for (int64_t k = *a; k < *b; ++k) {
      const int64_t c = col[k];
      if (c != r) atomicOr(&bits[(c - cb0) * (kMR / 32) + (tid >> 5)], 1u << (tid & 31));
    }
  }
  __syncthreads();
}

// Per upper tile: how many strictly-upper entries each of its 64 columns holds.
__global__ void __launch_bounds__(kMR) k_mir_colcounts(int64_t n, const int64_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col,
                                                       const int32_t* __restrict__ tile_rb,
                                                       const int32_t* __restrict__ tile_cb,
                                                       int32_t* __restrict__ cnt) {
  __shared__ unsigned bits[kMC * (kMR / 32)];
  const int64_t t = blockIdx.x;
  int64_t a, b;
  tile_bits(n, rowptr, col, (int64_t)tile_rb[t] * kMR, (int64_t)tile_cb[t] * kMC, bits, &a, &b);
  if (threadIdx.x < kMC) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < kMR / 32; ++w) s += __popc(bits[threadIdx.x * (kMR / 32) + w]);
    cnt[t * kMC + threadIdx.x] = s;
  }
}

// Thread per column c: offsets of each upper tile's contribution to row c's lower part (tiles of
// c's column block in ascending row-block order), and the lower-part length of row c.
__global__ void k_mir_coloffsets(int64_t n, const int64_t* __restrict__ jt_ptr, const int32_t* __restrict__ jt_tile,
                                 const int32_t* __restrict__ cnt, int32_t* __restrict__ off,
                                 int64_t* __restrict__ lower) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int64_t J = c / kMC;
  const int j = (int)(c - J * kMC);
  int64_t run = 0;
  for (int64_t p = jt_ptr[J]; p < jt_ptr[J + 1]; ++p) {
    const int64_t t = jt_tile[p];
    off[t * kMC + j] = (int32_t)run;
    run += cnt[t * kMC + j];
  }
  lower[c] = run;
}

// Row lengths of the mirrored matrix.
__global__ void k_mir_rowlen(int64_t n, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ lower,
                             int64_t* __restrict__ len) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) len[r] = lower[r] + rowptr[r + 1] - rowptr[r];
}

// Strict lower part: entry (r, c) of upper tile t goes to row c, after the contributions of
// earlier row blocks, at its rank among the tile's entries of column c (rows ascending).
template <typename V>
__global__ void __launch_bounds__(kMR) k_mir_lower(int64_t n, const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const V* __restrict__ val,
                                                   const int32_t* __restrict__ tile_rb,
                                                   const int32_t* __restrict__ tile_cb,
                                                   const int32_t* __restrict__ off,
                                                   const int64_t* __restrict__ fptr, int32_t* __restrict__ fcol,
                                                   V* __restrict__ fval) {
  __shared__ unsigned bits[kMC * (kMR / 32)];
  const int64_t t = blockIdx.x;
  const int64_t r0 = (int64_t)tile_rb[t] * kMR, cb0 = (int64_t)tile_cb[t] * kMC;
  int64_t a, b;
  tile_bits(n, rowptr, col, r0, cb0, bits, &a, &b);
  const int tid = threadIdx.x;
  const int64_t r = r0 + tid;
  const int w = tid >> 5;
  const unsigned below = (1u << (tid & 31)) - 1u;
  for (int64_t k = a; k < b; ++k) {
    const int64_t c = col[k];
    if (c == r) continue;
    const int j = (int)(c - cb0);
    const unsigned* bj = bits + j * (kMR / 32);
    int rank = __popc(bj[w] & below);
    for (int ww = 0; ww < w; ++ww) rank += __popc(bj[ww]);
    const int64_t pos = fptr[c] + off[t * kMC + j] + rank;
    fcol[pos] = (int32_t)r;
    fval[pos] = val[k];
  }
}

// Upper part (diagonal included) after the lower part of each row.
template <typename V>
__global__ void k_mir_upper(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const V* __restrict__ val, const int64_t* __restrict__ lower,
                            const int64_t* __restrict__ fptr, int32_t* __restrict__ fcol, V* __restrict__ fval) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t base = fptr[r] + lower[r] - rowptr[r];
  for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    fcol[base + k] = col[k];
    fval[base + k] = val[k];
  }
}

// Thread per row of the mirrored CSR: entries of the row in each tile of its row block.
__global__ void k_mir_rowtile_counts(int64_t n, const int64_t* __restrict__ fptr, const int32_t* __restrict__ fcol,
                                     const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ tile_col,
                                     uint8_t* __restrict__ cnt) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t I = r / kMR;
  const int rl = (int)(r - I * kMR);
  int64_t t = tile_ptr[I];
  const int64_t tend = tile_ptr[I + 1];
  int run = 0;
  int64_t tcur = -1;
  for (int64_t k = fptr[r]; k < fptr[r + 1]; ++k) {
    const int J = fcol[k] / kMC;
    while (t < tend && tile_col[t] < J) ++t;
    if (t != tcur) {
      if (tcur >= 0) cnt[tcur * kMR + rl] = (uint8_t)run;
      tcur = t;
      run = 0;
    }
    ++run;
  }
  if (tcur >= 0) cnt[tcur * kMR + rl] = (uint8_t)run;
}

// Thread per (tile, group): quads of the group = ceil(longest row / 4).
__global__ void k_mir_group_quads(int64_t n_tiles, const uint8_t* __restrict__ cnt, uint8_t* __restrict__ gq) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_tiles * kMGroups) return;
  int m = 0;
#pragma unroll
  for (int k = 0; k < kMG; ++k) m = max(m, (int)cnt[i * kMG + k]);
  gq[i] = (uint8_t)((m + 3) / 4);
}

// Thread per row: scatter the row's entries of every tile into its group's quads.
template <typename V>
__global__ void k_mir_scatter(int64_t n, const int64_t* __restrict__ fptr, const int32_t* __restrict__ fcol,
                              const V* __restrict__ fval, const int64_t* __restrict__ tile_ptr,
                              const int32_t* __restrict__ tile_col, const int64_t* __restrict__ gdst,
                              uint8_t* __restrict__ mcol, V* __restrict__ mval) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t I = r / kMR;
  const int rl = (int)(r - I * kMR);
  const int g = rl / kMG, i = rl % kMG;
  int64_t t = tile_ptr[I];
  const int64_t tend = tile_ptr[I + 1];
  int64_t tcur = -1, base = 0;
  int kk = 0;
  for (int64_t k = fptr[r]; k < fptr[r + 1]; ++k) {
    const int c = fcol[k];
    const int J = c / kMC;
    while (t < tend && tile_col[t] < J) ++t;
    if (t != tcur) {
      tcur = t;
      base = gdst[t * kMGroups + g];
      kk = 0;
    }
    const int64_t slot = base + (int64_t)(kk >> 2) * 32 + i * 4 + (kk & 3);
    mcol[slot] = (uint8_t)(c - J * kMC);
    mval[slot] = fval[k];
    ++kk;
  }
}

template <typename V>
eig_status mirror_fill(SpmmPlan* P, const int32_t* tile_rb, const int32_t* tile_cb, int64_t n_up_tiles,
                       const int64_t* jt_ptr, const int32_t* jt_tile, int capq, cudaStream_t st) {
  const int64_t n = P->n;
  const int tb = 256;
  const int64_t gb = (n + tb - 1) / tb;
  const V* val = static_cast<const V*>(P->val);
  // 1. lower-part lengths and offsets
  DevBuf cnt, off, lower, fptr;
  EIG_TRY(cnt.reserve(std::max<int64_t>(n_up_tiles, 1) * kMC * 4));
  EIG_TRY(off.reserve(std::max<int64_t>(n_up_tiles, 1) * kMC * 4));
  EIG_TRY(lower.reserve(n * 8));
  EIG_TRY(fptr.reserve((n + 1) * 8));
  if (n_up_tiles) {
    k_mir_colcounts<<<(unsigned)n_up_tiles, kMR, 0, st>>>(n, P->rowptr, P->col, tile_rb, tile_cb, cnt.as<int32_t>());
    EIG_LAUNCH_CHECK("k_mir_colcounts");
  }
  k_mir_coloffsets<<<(unsigned)gb, tb, 0, st>>>(n, jt_ptr, jt_tile, cnt.as<int32_t>(), off.as<int32_t>(),
                                                lower.as<int64_t>());
  EIG_LAUNCH_CHECK("k_mir_coloffsets");
  k_mir_rowlen<<<(unsigned)gb, tb, 0, st>>>(n, P->rowptr, lower.as<int64_t>(), fptr.as<int64_t>());
  EIG_LAUNCH_CHECK("k_mir_rowlen");
  std::vector<int64_t> h_len(n), h_fptr(n + 1, 0);
  EIG_CUDA_TRY(cudaMemcpyAsync(h_len.data(), fptr.p, n * 8, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t r = 0; r < n; ++r) h_fptr[r + 1] = h_fptr[r] + h_len[r];
  const int64_t fnnz = h_fptr[n];
  P->m_full_nnz = fnnz;
  EIG_CUDA_TRY(cudaMemcpyAsync(fptr.p, h_fptr.data(), (n + 1) * 8, cudaMemcpyHostToDevice, st));
  // 2. the mirrored CSR
  DevBuf fcol, fval;
  EIG_TRY(fcol.reserve(std::max<int64_t>(fnnz, 1) * 4));
  EIG_TRY(fval.reserve(std::max<int64_t>(fnnz, 1) * sizeof(V)));
  if (n_up_tiles) {
    k_mir_lower<V><<<(unsigned)n_up_tiles, kMR, 0, st>>>(n, P->rowptr, P->col, val, tile_rb, tile_cb,
                                                         off.as<int32_t>(), fptr.as<int64_t>(), fcol.as<int32_t>(),
                                                         fval.as<V>());
    EIG_LAUNCH_CHECK("k_mir_lower");
  }
  k_mir_upper<V><<<(unsigned)gb, tb, 0, st>>>(n, P->rowptr, P->col, val, lower.as<int64_t>(), fptr.as<int64_t>(),
                                              fcol.as<int32_t>(), fval.as<V>());
  EIG_LAUNCH_CHECK("k_mir_upper");
  cnt.release();
  off.release();
  lower.release();
  // 3. tiles of the mirrored matrix and their group quad counts
  DevBuf ftile_ptr, ftile_col;
  std::vector<int64_t> h_tptr;
  std::vector<int32_t> h_tcol;
  EIG_TRY(build_tile_lists(n, kMR, kMC, fptr.as<int64_t>(), fcol.as<int32_t>(), st, ftile_ptr, ftile_col, h_tptr,
                           h_tcol));
  const int64_t nRB = (n + kMR - 1) / kMR;
  const int64_t nt = h_tptr[nRB];
  DevBuf rcnt, gq;
  EIG_TRY(rcnt.reserve(std::max<int64_t>(nt, 1) * kMR));
  EIG_TRY(gq.reserve(std::max<int64_t>(nt, 1) * kMGroups));
  EIG_CUDA_TRY(cudaMemsetAsync(rcnt.p, 0, std::max<int64_t>(nt, 1) * kMR, st));
  k_mir_rowtile_counts<<<(unsigned)gb, tb, 0, st>>>(n, fptr.as<int64_t>(), fcol.as<int32_t>(),
                                                     ftile_ptr.as<int64_t>(), ftile_col.as<int32_t>(),
                                                     rcnt.as<uint8_t>());
  EIG_LAUNCH_CHECK("k_mir_rowtile_counts");
  if (nt) {
    k_mir_group_quads<<<(unsigned)((nt * kMGroups + tb - 1) / tb), tb, 0, st>>>(nt, rcnt.as<uint8_t>(),
                                                                             gq.as<uint8_t>());
    EIG_LAUNCH_CHECK("k_mir_group_quads");
  }
  std::vector<uint8_t> h_gq((size_t)nt * kMGroups);
  if (nt) EIG_CUDA_TRY(cudaMemcpyAsync(h_gq.data(), gq.p, (size_t)nt * kMGroups, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  rcnt.release();
  gq.release();
  // 4. chunks: runs of consecutive groups of one tile holding at most capq quads
  std::vector<MirrorChunk> ch;
  std::vector<uint8_t> cgq;
  std::vector<int64_t> cptr(nRB + 1, 0);
  std::vector<int64_t> gdst((size_t)nt * kMGroups, 0);
  int64_t slots = 0;
  for (int64_t I = 0; I < nRB; ++I) {
    for (int64_t t = h_tptr[I]; t < h_tptr[I + 1]; ++t) {
      const uint8_t* q = h_gq.data() + (size_t)t * kMGroups;
      int g = 0;
      while (g < kMGroups) {
        MirrorChunk k;
        k.ent_off = slots;
        k.J = h_tcol[t];
        k.g0 = g;
        int nq = 0;
        uint8_t tab[kMGroups] = {0};
        while (g < kMGroups && (nq + q[g] <= capq || g == k.g0)) {
          gdst[(size_t)t * kMGroups + g] = slots + (int64_t)nq * 32;
          tab[g] = q[g];
          nq += q[g];
          ++g;
        }
        k.g1 = g;
        k.nq = nq;
        k.pad = 0;
        if (nq == 0) continue;  // groups without entries (cannot end a tile with entries)
        slots += (int64_t)nq * 32;
        ch.push_back(k);
        cgq.insert(cgq.end(), tab, tab + kMGroups);
      }
    }
    cptr[I + 1] = (int64_t)ch.size();
  }
  P->m_nchunks = (int64_t)ch.size();
  P->m_slots = slots;
  P->m_capq = capq;
  EIG_TRY(P->m_chunk_ptr.reserve((nRB + 1) * 8));
  EIG_TRY(P->m_chunks.reserve(std::max<size_t>(ch.size(), 1) * sizeof(MirrorChunk)));
  EIG_TRY(P->m_gq.reserve(std::max<size_t>(cgq.size(), 32)));
  EIG_TRY(P->m_col.reserve(std::max<int64_t>(slots, 32)));
  EIG_TRY(P->m_val.reserve(std::max<int64_t>(slots, 32) * sizeof(V)));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->m_chunk_ptr.p, cptr.data(), (nRB + 1) * 8, cudaMemcpyHostToDevice, st));
  if (!ch.empty()) {
    EIG_CUDA_TRY(cudaMemcpyAsync(P->m_chunks.p, ch.data(), ch.size() * sizeof(MirrorChunk), cudaMemcpyHostToDevice,
                                 st));
    EIG_CUDA_TRY(cudaMemcpyAsync(P->m_gq.p, cgq.data(), cgq.size(), cudaMemcpyHostToDevice, st));
  }
  EIG_CUDA_TRY(cudaMemsetAsync(P->m_col.p, (int)kPadCol, std::max<int64_t>(slots, 32), st));
  EIG_CUDA_TRY(cudaMemsetAsync(P->m_val.p, 0, std::max<int64_t>(slots, 32) * sizeof(V), st));
  DevBuf dgdst;
  EIG_TRY(dgdst.reserve(std::max<size_t>(gdst.size(), 1) * 8));
  if (!gdst.empty())
    EIG_CUDA_TRY(cudaMemcpyAsync(dgdst.p, gdst.data(), gdst.size() * 8, cudaMemcpyHostToDevice, st));
  k_mir_scatter<V><<<(unsigned)gb, tb, 0, st>>>(n, fptr.as<int64_t>(), fcol.as<int32_t>(), fval.as<V>(),
                                                ftile_ptr.as<int64_t>(), ftile_col.as<int32_t>(),
                                                dgdst.as<int64_t>(), P->m_col.as<uint8_t>(), P->m_val.as<V>());
  EIG_LAUNCH_CHECK("k_mir_scatter");
  EIG_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors and temporaries go out of scope
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------------------
struct MirrorArgs {
  int64_t n;
  int capq;
  const int64_t* chunk_ptr;
  const MirrorChunk* chunks;
  const uint8_t* mcol;
  const void* mval;
  const uint8_t* mgq;
  int* err;
};

__host__ __device__ constexpr size_t al128(size_t b) { return (b + 127) & ~size_t(127); }

// Byte offsets inside one pipeline stage.
struct MirrorStage {
  size_t col, val, gq, xj, bytes;
  __host__ __device__ MirrorStage(int capq, int vbytes, int rowbytes) {
    col = 0;
    val = al128((size_t)capq * 32);
    gq = val + al128((size_t)capq * 32 * vbytes);
    xj = gq + 128;
    bytes = xj + al128((size_t)kMC * rowbytes);
  }
};

// Four consecutive values of a quad row, widened to the arithmetic type.
template <typename V, typename T> struct QuadLoad;
template <typename T> struct QuadLoad<float, T> {
  __device__ __forceinline__ static void ld(const float* p, T (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = (T)a.x; v[1] = (T)a.y; v[2] = (T)a.z; v[3] = (T)a.w;
  }
};
template <typename T> struct QuadLoad<uint16_t, T> {
  __device__ __forceinline__ static void ld(const uint16_t* p, T (&v)[4]) {
    const uint2 a = *reinterpret_cast<const uint2*>(p);
    v[0] = (T)__uint_as_float(a.x << 16);
    v[1] = (T)__uint_as_float(a.x & 0xFFFF0000u);
    v[2] = (T)__uint_as_float(a.y << 16);
    v[3] = (T)__uint_as_float(a.y & 0xFFFF0000u);
  }
};
template <typename T> struct QuadLoad<double, T> {
  __device__ __forceinline__ static void ld(const double* p, T (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = (T)a.x; v[1] = (T)a.y; v[2] = (T)b.x; v[3] = (T)b.y;
  }
};

template <typename T>
__device__ __forceinline__ T pick4(const T (&v)[4], int j) {
  T r = v[0];
  r = (j == 1) ? v[1] : r;
  r = (j == 2) ? v[2] : r;
  r = (j == 3) ? v[3] : r;
  return r;
}

// Accumulation of y += v * x over one lane's EPL elements.
//   Plain: X rows staged as T, fma in T.
//   DF (FP64 vectors with FP32 or BF16 values): X rows staged as (hi, lo) FP32 pairs (same 8 bytes
//   per element as FP64), each product taken exactly (hi part by an FMA-based two-product, lo part
//   rounded) and summed in double-float (two-sum into hi, errors into lo): ~2^-44 relative per
//   step, at FP32 instruction rate instead of the much slower FP64 pipe of sm_103a.
template <bool DF, typename T, int EPL> struct MirrorAcc;
template <typename T, int EPL> struct MirrorAcc<false, T, EPL> {
  typedef T VT;   // value type in arithmetic
  typedef Vec<T, EPL> XV;
  Vec<T, EPL> y;
  __device__ __forceinline__ void zero() { y.zero(); }
  __device__ __forceinline__ static XV load(const unsigned char* p) {
    return VecIO<T, EPL>::ld(reinterpret_cast<const T*>(p));
  }
  __device__ __forceinline__ void add(T v, const XV& x) {
#pragma unroll
    for (int e = 0; e < EPL; ++e) y.v[e] = fma(v, x.v[e], y.v[e]);
  }
  __device__ __forceinline__ T get(int e) const { return y.v[e]; }
  // staged form of one element
  __device__ __forceinline__ static void stage(const T* src, unsigned char* dst) {
    VecIO<T, EPL>::st(reinterpret_cast<T*>(dst), VecIO<T, EPL>::ld(src));
  }
  __device__ __forceinline__ static void stage_zero(unsigned char* dst) {
    Vec<T, EPL> z;
    z.zero();
    VecIO<T, EPL>::st(reinterpret_cast<T*>(dst), z);
  }
};
template <int EPL> struct MirrorAcc<true, double, EPL> {
  typedef float VT;
  struct XV { float h[EPL], l[EPL]; };
  float hi[EPL], lo[EPL];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int e = 0; e < EPL; ++e) hi[e] = lo[e] = 0.0f;
  }
  __device__ __forceinline__ static XV load(const unsigned char* p) {
    XV x;
    if (EPL == 2) {
      const float4 a = *reinterpret_cast<const float4*>(p);
      x.h[0] = a.x; x.l[0] = a.y; x.h[EPL - 1] = a.z; x.l[EPL - 1] = a.w;
    } else {
      const float2 a = *reinterpret_cast<const float2*>(p);
      x.h[0] = a.x; x.l[0] = a.y;
    }
    return x;
  }
  __device__ __forceinline__ void add(float v, const XV& x) {
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const float p = v * x.h[e];
      const float pe = fmaf(v, x.h[e], -p);          // v * x.h[e] = p + pe exactly
      const float s = hi[e] + p;
      const float bb = s - hi[e];
      const float err = (hi[e] - (s - bb)) + (p - bb);  // hi + p = s + err exactly
      hi[e] = s;
      lo[e] = fmaf(v, x.l[e], lo[e] + (err + pe));
    }
  }
  __device__ __forceinline__ double get(int e) const { return (double)hi[e] + (double)lo[e]; }
  __device__ __forceinline__ static void stage(const double* src, unsigned char* dst) {
    float* d = reinterpret_cast<float*>(dst);
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const double x = src[e];
      const float h = __double2float_rn(x);
      d[2 * e] = h;
      d[2 * e + 1] = __double2float_rn(x - (double)h);
    }
  }
  __device__ __forceinline__ static void stage_zero(unsigned char* dst) {
    float* d = reinterpret_cast<float*>(dst);
#pragma unroll
    for (int e = 0; e < 2 * EPL; ++e) d[e] = 0.0f;
  }
};

// Double-float accumulation applies to FP64 vectors with FP32 or BF16 values.
template <typename T, typename V> struct MirrorDF { static constexpr bool value = false; };
template <> struct MirrorDF<double, float> { static constexpr bool value = true; };
template <> struct MirrorDF<double, uint16_t> { static constexpr bool value = true; };

// Launch shape of the kernel for (T, NB).
template <typename T, int NB> struct MirrorShape {
  typedef LaneShape<T, NB> S;
  static constexpr int EPL = S::EPL, L = S::L;
  static constexpr int P = 32 / L;                    // slots per warp instruction
  static constexpr int RPI = P < kMG ? P : kMG;       // rows of a group per instruction
  static constexpr int SB = kMG / RPI;                // row sub-blocks of a group
  static constexpr int M = P / RPI;                   // steps of a quad per instruction
  static constexpr int JJ = 4 / M;                    // steps of a quad per lane
  static constexpr int RB = NB * (int)sizeof(T);      // bytes of one X row
  static constexpr int NCOPY = RB < 128 ? 128 / RB : 1;
  static constexpr int LINE = RB < 128 ? 128 : RB;    // bytes of one replicated X row
  // registers of y per lane with 4 warps (32-bit words); more warps when it is large
  static constexpr int YREG4 = (kMGroups / 4) * SB * EPL * (int)sizeof(T) / 4;
  // 4 warps for FP32 vectors (measured fastest); 8 for FP64-sized elements, whose
  // double-float or FP64 arithmetic gains from more resident warps
  static constexpr int WARPS = (sizeof(T) == 8 || YREG4 > 48) ? 8 : 4;
  static constexpr int MINB = WARPS == 4 ? 2 : (YREG4 > 48 ? 2 : 3);   // resident CTAs aimed for
  static constexpr int GPW = kMGroups / WARPS;
};

// Fused epilogue of a Chebyshev step (Alg. 3, Eq. chebypoly): Y = a (H X - c X) - Qp (first: no
// Qp), and Y = X on inactive (locked) columns; the same double arithmetic on the same rounded
// product H X as the separate elementwise pass.
struct MirrorEpi {
  const void* Qp;
  const int* active;
  double a, c;
  int first;
};

template <typename T, typename V, int NB, bool CHEB = false>
__global__ void __launch_bounds__(MirrorShape<T, NB>::WARPS * 32, MirrorShape<T, NB>::MINB)
k_spmm_mirror(MirrorArgs a, const T* __restrict__ X, T* __restrict__ Y, int xj_bulk, MirrorEpi epi) {
  typedef MirrorShape<T, NB> Sh;
  constexpr int EPL = Sh::EPL, L = Sh::L, RPI = Sh::RPI, SB = Sh::SB, M = Sh::M, JJ = Sh::JJ;
  constexpr int RB = Sh::RB, NCOPY = Sh::NCOPY, LINE = Sh::LINE, WARPS = Sh::WARPS, GPW = Sh::GPW;
  constexpr int NT = WARPS * 32;
  static_assert(M * JJ == 4, "quad split");
  typedef typename ValLoad<V>::storage VS;
  constexpr bool DF = MirrorDF<T, V>::value;
  typedef MirrorAcc<DF, T, EPL> Acc;
  typedef typename Acc::VT AT;
  extern __shared__ __align__(128) unsigned char smem[];
  const MirrorStage SL(a.capq, (int)sizeof(VS), RB);
  unsigned char* stage[2] = {smem, smem + SL.bytes};
  unsigned char* dup = smem + 2 * SL.bytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(dup + (size_t)kMC * LINE);
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t I = blockIdx.x;
  const int64_t r0 = I * kMR;
  const int slot = lane / L, q = lane % L;
  const int rsub = slot % RPI, sp = slot / RPI, cpy = slot % NCOPY;
  const int64_t c0 = a.chunk_ptr[I], c1 = a.chunk_ptr[I + 1];
  const VS* mval = static_cast<const VS*>(a.mval);

  Acc y[GPW][SB];
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi)
#pragma unroll
    for (int sb = 0; sb < SB; ++sb) y[gi][sb].zero();

  if (tid == 0) {
    s_abort = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();

  auto issue = [&](int64_t k, int s) {
    const MirrorChunk ck = a.chunks[k];
    const int64_t cb0 = (int64_t)ck.J * kMC;
    const int64_t avail = min64(kMC, a.n - cb0);
    const uint32_t cb = (uint32_t)ck.nq * 32u;
    const uint32_t vb = cb * (uint32_t)sizeof(VS);
    const uint32_t xb = xj_bulk ? (uint32_t)(avail * RB) : 0u;
    mbar_arrive_expect_tx(&bar[s], cb + vb + 32u + xb);
    unsigned char* st = stage[s];
    tma_load_1d(st + SL.col, a.mcol + ck.ent_off, cb, &bar[s]);
    tma_load_1d(st + SL.val, mval + ck.ent_off, vb, &bar[s]);
    tma_load_1d(st + SL.gq, a.mgq + k * kMGroups, 32u, &bar[s]);
    if (xj_bulk) tma_load_1d(st + SL.xj, X + cb0 * NB, xb, &bar[s]);
  };
  int issued[2] = {0, 0}, consumed[2] = {0, 0};  // meaningful in thread 0 only
  if (tid == 0) {
    if (c0 < c1) { issue(c0, 0); issued[0]++; }
    if (c0 + 1 < c1) { issue(c0 + 1, 1); issued[1]++; }
  }
  // X rows are read from the replicated lines, or straight from the staged copy when one row
  // already spans a whole bank line
  constexpr bool kDup = NCOPY > 1 || DF;
  int64_t prevJ = -1;
  for (int64_t k = c0; k < c1; ++k) {
    const int s = (int)((k - c0) & 1);
    const uint32_t phase = (uint32_t)(((k - c0) >> 1) & 1);
    const MirrorChunk ck = a.chunks[k];
    const int64_t cb0 = (int64_t)ck.J * kMC;
    const int64_t avail = min64(kMC, a.n - cb0);
    unsigned char* st = stage[s];
    if (!mbar_wait_bounded(&bar[s], phase)) {
      atomicOr(a.err, 1);
      s_abort = 1;
    }
    if (tid == 0) consumed[s]++;
    __syncthreads();
    if (s_abort) break;
    const T* xsrc;
    if (kDup || !xj_bulk) {
      // replicate X_J (zero rows past n) unless this chunk continues the previous tile
      if (ck.J != prevJ) {
        const T* sxj = reinterpret_cast<const T*>(st + SL.xj);
        for (int e = tid; e < kMC * NB / EPL; e += NT) {
          const int c = (e * EPL) / NB, o = (e * EPL) % NB;
          const T* src = xj_bulk ? sxj + c * NB + o : X + (cb0 + c) * NB + o;
#pragma unroll
          for (int p = 0; p < NCOPY; ++p) {
            unsigned char* dst = dup + (size_t)c * LINE + (size_t)p * RB + (size_t)o * sizeof(T);
            if (c < avail) Acc::stage(src, dst);
            else Acc::stage_zero(dst);
          }
        }
        __syncthreads();
      }
      xsrc = reinterpret_cast<const T*>(dup);
    } else {
      // staged rows past n are never read: their columns do not occur
      xsrc = reinterpret_cast<const T*>(st + SL.xj);
    }
    prevJ = ck.J;
    const uint8_t* scol = st + SL.col;
    const VS* sval = reinterpret_cast<const VS*>(st + SL.val);
    // quad offsets of the chunk's groups: exclusive prefix of the 32 counts
    const int gcount = st[SL.gq + lane];
    int incl = gcount;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int excl = incl - gcount;
    const unsigned char* xbase = reinterpret_cast<const unsigned char*>(xsrc) + (size_t)cpy * (kDup ? RB : 0) +
                                 (size_t)q * EPL * sizeof(T);
#pragma unroll
    for (int gi = 0; gi < GPW; ++gi) {
      const int g = gi * WARPS + w;
      const int nq = __shfl_sync(0xffffffffu, gcount, g);
      const int qo = __shfl_sync(0xffffffffu, excl, g);
#pragma unroll
      for (int sb = 0; sb < SB; ++sb) {
        const int i = rsub + sb * RPI;
        for (int qq = 0; qq < nq; ++qq) {
          const int base = (qo + qq) * 32 + i * 4;
          const uint32_t cq = *reinterpret_cast<const uint32_t*>(scol + base);
          AT vq[4];
          QuadLoad<VS, AT>::ld(sval + base, vq);
#pragma unroll
          for (int jj = 0; jj < JJ; ++jj) {
            const int j = (M == 1) ? jj : sp + jj * M;
            const unsigned c = (cq >> (8 * j)) & 0xFFu;
            const AT v = (M == 1) ? vq[jj] : pick4(vq, j);
            if (c != kPadCol) y[gi][sb].add(v, Acc::load(xbase + (size_t)c * LINE));
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && k + 2 < c1) {
      fence_proxy_async();
      issue(k + 2, s);
      issued[s]++;
    }
  }
  if (s_abort) {
    // leave no bulk copy in flight into this CTA's shared memory (bounded waits)
    if (tid == 0)
      for (int ss = 0; ss < 2; ++ss)
        while (consumed[ss] < issued[ss]) {
          if (!mbar_wait_bounded(&bar[ss], (uint32_t)(consumed[ss] & 1))) break;
          consumed[ss]++;
        }
    __syncthreads();
    return;
  }
  // combine the step phases of each row (fixed xor tree), then one store per row slice
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi) {
    const int g = gi * WARPS + w;
#pragma unroll
    for (int sb = 0; sb < SB; ++sb) {
      Vec<T, EPL> out;
#pragma unroll
      for (int e = 0; e < EPL; ++e) {
        T v = y[gi][sb].get(e);
#pragma unroll
        for (int o = RPI * L; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        out.v[e] = v;
      }
      const int64_t r = r0 + g * kMG + rsub + sb * RPI;
      if (CHEB && sp == 0 && r < a.n) {
        const T* Qp = static_cast<const T*>(epi.Qp);
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int jc = q * EPL + e;
          const T wv = X[r * NB + jc];
          if (!epi.active[jc]) {
            out.v[e] = wv;
          } else {
            double yv = epi.a * ((double)out.v[e] - epi.c * (double)wv);
            if (!epi.first) yv -= (double)Qp[r * NB + jc];
            out.v[e] = (T)yv;
          }
        }
      }
      if (sp == 0 && r < a.n) VecIO<T, EPL>::st(Y + r * NB + q * EPL, out);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
size_t mirror_bytes_estimate(const SpmmPlan* P) {
  // mirrored CSR (temporary) + quads with ~1.5x padding
  const double fnnz = 2.0 * double(P->nnz);
  const double vb = double(dtype_size(P->val_type));
  return (size_t)(fnnz * (4.0 + vb) + 1.6 * fnnz * (1.0 + vb) + 64.0 * double(P->n));
}

eig_status spmm_plan_build_mirror(SpmmPlan* P, const std::vector<int64_t>& h_tptr,
                                  const std::vector<int32_t>& h_tcol, cudaStream_t st) {
  if (P->R != kMR || P->C != kMC) return EIG_EUNSUPPORTED;
  const int64_t nRB = P->nRB, nCB = P->nCB, nt = P->n_tiles;
  // row block of each upper tile, and the upper tiles grouped by column block (ascending row block)
  std::vector<int32_t> trb(std::max<int64_t>(nt, 1)), tcb(std::max<int64_t>(nt, 1));
  std::vector<int64_t> jptr(nCB + 1, 0);
  for (int64_t I = 0; I < nRB; ++I)
    for (int64_t t = h_tptr[I]; t < h_tptr[I + 1]; ++t) {
      trb[t] = (int32_t)I;
      tcb[t] = h_tcol[t];
      jptr[h_tcol[t] + 1]++;
    }
  for (int64_t J = 0; J < nCB; ++J) jptr[J + 1] += jptr[J];
  std::vector<int32_t> jt(std::max<int64_t>(nt, 1));
  {
    std::vector<int64_t> fill(jptr.begin(), jptr.end() - 1);
    for (int64_t t = 0; t < nt; ++t) jt[fill[tcb[t]]++] = (int32_t)t;
  }
  DevBuf d_trb, d_tcb, d_jptr, d_jt;
  EIG_TRY(d_trb.reserve(trb.size() * 4));
  EIG_TRY(d_tcb.reserve(tcb.size() * 4));
  EIG_TRY(d_jptr.reserve(jptr.size() * 8));
  EIG_TRY(d_jt.reserve(jt.size() * 4));
  EIG_CUDA_TRY(cudaMemcpyAsync(d_trb.p, trb.data(), trb.size() * 4, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(d_tcb.p, tcb.data(), tcb.size() * 4, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(d_jptr.p, jptr.data(), jptr.size() * 8, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(d_jt.p, jt.data(), jt.size() * 4, cudaMemcpyHostToDevice, st));
  // stage payload ~18 KB of quads
  const int vb = (int)dtype_size(P->val_type);
  const int capq = std::max(16, 18432 / (32 * (1 + vb)));
  eig_status s;
  if (P->val_type == EIG_F32)
    s = mirror_fill<float>(P, d_trb.as<int32_t>(), d_tcb.as<int32_t>(), nt, d_jptr.as<int64_t>(), d_jt.as<int32_t>(),
                           capq, st);
  else if (P->val_type == EIG_F64)
    s = mirror_fill<double>(P, d_trb.as<int32_t>(), d_tcb.as<int32_t>(), nt, d_jptr.as<int64_t>(),
                            d_jt.as<int32_t>(), capq, st);
  else
    s = mirror_fill<uint16_t>(P, d_trb.as<int32_t>(), d_tcb.as<int32_t>(), nt, d_jptr.as<int64_t>(),
                              d_jt.as<int32_t>(), capq, st);
  EIG_TRY(s);
  if (!P->err.p) {
    EIG_TRY(P->err.reserve(16));
    EIG_CUDA_TRY(cudaMemsetAsync(P->err.p, 0, 16, st));
    EIG_CUDA_TRY(cudaStreamSynchronize(st));
  }
  P->mirrored = true;
  return EIG_OK;
}

template <typename T, typename V, int NB>
static size_t mirror_smem(const SpmmPlan* P) {
  typedef MirrorShape<T, NB> Sh;
  const MirrorStage SL(P->m_capq, (int)sizeof(typename ValLoad<V>::storage), Sh::RB);
  return 2 * SL.bytes + (size_t)kMC * Sh::LINE + 2 * 8;
}

template <typename T, typename V, int NB>
eig_status mirror_launch(SpmmPlan* P, const T* X, T* Y, cudaStream_t st) {
  typedef MirrorShape<T, NB> Sh;
  int dev = 0, maxsm = 0;
  EIG_CUDA_TRY(cudaGetDevice(&dev));
  EIG_CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t sm = mirror_smem<T, V, NB>(P);
  if (sm > (size_t)maxsm) return EIG_EUNSUPPORTED;
  MirrorArgs a;
  a.n = P->n;
  a.capq = P->m_capq;
  a.chunk_ptr = P->m_chunk_ptr.as<int64_t>();
  a.chunks = P->m_chunks.as<MirrorChunk>();
  a.mcol = P->m_col.as<uint8_t>();
  a.mval = P->m_val.p;
  a.mgq = P->m_gq.as<uint8_t>();
  a.err = P->err.as<int>();
  // X_J by bulk copy needs 16-byte aligned rows of a 16-byte multiple
  const int xj_bulk = (Sh::RB % 16 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
  auto kern = k_spmm_mirror<T, V, NB>;
  EIG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<(unsigned)P->nRB, Sh::WARPS * 32, sm, st>>>(a, X, Y, xj_bulk, MirrorEpi());
  EIG_LAUNCH_CHECK("k_spmm_mirror");
  return EIG_OK;
}

// The Chebyshev-step variant (same kernel, fused epilogue).
template <typename T, typename V, int NB>
eig_status mirror_launch_cheb(SpmmPlan* P, const T* X, T* Y, const T* Qp, const int* active, double alpha, double c,
                              int first, cudaStream_t st) {
  typedef MirrorShape<T, NB> Sh;
  int dev = 0, maxsm = 0;
  EIG_CUDA_TRY(cudaGetDevice(&dev));
  EIG_CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t sm = mirror_smem<T, V, NB>(P);
  if (sm > (size_t)maxsm) return EIG_EUNSUPPORTED;
  MirrorArgs a;
  a.n = P->n;
  a.capq = P->m_capq;
  a.chunk_ptr = P->m_chunk_ptr.as<int64_t>();
  a.chunks = P->m_chunks.as<MirrorChunk>();
  a.mcol = P->m_col.as<uint8_t>();
  a.mval = P->m_val.p;
  a.mgq = P->m_gq.as<uint8_t>();
  a.err = P->err.as<int>();
  MirrorEpi epi;
  epi.Qp = Qp;
  epi.active = active;
  epi.a = alpha;
  epi.c = c;
  epi.first = first;
  const int xj_bulk = (Sh::RB % 16 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
  auto kern = k_spmm_mirror<T, V, NB, true>;
  EIG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  kern<<<(unsigned)P->nRB, Sh::WARPS * 32, sm, st>>>(a, X, Y, xj_bulk, epi);
  EIG_LAUNCH_CHECK("k_spmm_mirror_cheb");
  return EIG_OK;
}

#define EIG_MIRROR_CHEB_INST(T, V)                                                                               \
  template eig_status mirror_launch_cheb<T, V, 8>(SpmmPlan*, const T*, T*, const T*, const int*, double, double,  \
                                                  int, cudaStream_t);                                            \
  template eig_status mirror_launch_cheb<T, V, 16>(SpmmPlan*, const T*, T*, const T*, const int*, double, double, \
                                                   int, cudaStream_t);                                           \
  template eig_status mirror_launch_cheb<T, V, 32>(SpmmPlan*, const T*, T*, const T*, const int*, double, double, \
                                                   int, cudaStream_t);
EIG_MIRROR_CHEB_INST(float, float)
EIG_MIRROR_CHEB_INST(double, double)
EIG_MIRROR_CHEB_INST(double, float)

#define EIG_MIRROR_INST(T, V)                                                           \
  template eig_status mirror_launch<T, V, 1>(SpmmPlan*, const T*, T*, cudaStream_t);    \
  template eig_status mirror_launch<T, V, 2>(SpmmPlan*, const T*, T*, cudaStream_t);    \
  template eig_status mirror_launch<T, V, 4>(SpmmPlan*, const T*, T*, cudaStream_t);    \
  template eig_status mirror_launch<T, V, 8>(SpmmPlan*, const T*, T*, cudaStream_t);    \
  template eig_status mirror_launch<T, V, 16>(SpmmPlan*, const T*, T*, cudaStream_t);   \
  template eig_status mirror_launch<T, V, 32>(SpmmPlan*, const T*, T*, cudaStream_t);
EIG_MIRROR_INST(float, float)
EIG_MIRROR_INST(float, uint16_t)
EIG_MIRROR_INST(double, double)
EIG_MIRROR_INST(double, float)
EIG_MIRROR_INST(double, uint16_t)

}  // namespace eig
