// Mirrored row-stream SpMM: Y = H X with H = U + U_strict^T given by its stored upper triangle U
// (Sec. 1; Eqs. upd1-upd2; the half storage of Sec. 3.1 is the input format), GB300 layout.
//
// Why mirror.  In a half-stored kernel every stored h_ij feeds a gather y_i += h_ij x_j and a
// scatter z_j += h_ij x_i; on sm_103a both run out of shared memory and the scatter costs a
// read-modify-write of an nb-wide row per nonzero.  Here the plan expands U once, on the
// device, into both triangles, so the kernel only gathers.
//
// What bounds it.  Every entry of H costs one gather of an nb-wide X row from shared memory
// (64 bytes at nb = 16 in FP32), so at nb >= 16 the shared-memory pipe (128 bytes per clock
// per SM), not HBM, is the limit; at nb <= 8 it is HBM.  The layout is built so that the pipe
// moves little else and never stalls on bank conflicts, and so that HBM sees enough bytes in
// flight:
//   * one lane owns one row: per row block (256 rows, one CTA of 8 warps) and per panel of
//     column tiles, the rows are ranked by their entry count and warp w's lane l takes the
//     row of rank 32 w + l; the warp steps through its longest row's count, shorter rows
//     padded with zero-valued entries (a few percent);
//   * each step, lane l gathers its entry's whole X row in 16-byte pieces, starting at a
//     lane-dependent piece, and the entries are ordered so that lane l reads a row of class
//     (l + step) mod 8 (X row index mod 8): the 8 lanes of every shared-memory phase then hit
//     distinct banks for any nb;
//   * the entries (uint16 panel-local column + value) stream from HBM straight into registers,
//     several 8-step blocks ahead, bypassing L1 and evicted first from L2; each lane loads
//     only its own entries (16 + 32 bytes per block in FP32), so nothing is loaded twice;
//   * X: the X rows of the row block's column tiles (64 rows each) are staged in shared
//     memory by bulk copies (TMA) in panels of at most 24 tiles, evicted last from L2; a row
//     block whose tiles do not fit takes several panels, its rows' partial sums added in Y
//     in panel order.
// Every sum runs in a fixed order (steps in stream order, panels in order): Y is bitwise
// reproducible.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "spmm.cuh"
#include "tma.cuh"
#include "vec.cuh"

namespace eig {

namespace {

constexpr int kMR = 256;                 // rows per row block (one CTA)
constexpr int kMC = 64;                  // columns per tile (unit of X staging)
constexpr int kW = 8;                    // warps per CTA; warp w takes the rows of rank [32 w, 32 w + 32)
constexpr int kRW = kMR / kW;            // rows per warp
constexpr int kBS = 8;                   // steps per streamed block
constexpr int kBE = 32 * kBS;            // entries per block (32 lanes)
constexpr int kPT = 24;                  // tiles per panel at most
constexpr int kPR = kPT * kMC;           // staged X rows per panel; 8 zero rows follow
constexpr int kL2 = 6;                   // streamed blocks prefetched into L2 ahead of use

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

// Upper part (diagonal included) after the lower part of each row.  Warp per row: the lanes
// copy consecutive entries.
template <typename V>
__global__ void k_mir_upper(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const V* __restrict__ val, const int64_t* __restrict__ lower,
                            const int64_t* __restrict__ fptr, int32_t* __restrict__ fcol, V* __restrict__ fval) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n) return;
  const int64_t k0 = rowptr[r], k1 = rowptr[r + 1];
  const int64_t base = fptr[r] + lower[r] - k0;
  for (int64_t k = k0 + lane; k < k1; k += 32) {
    fcol[base + k] = col[k];
    fval[base + k] = val[k];
  }
}

// ---------------------------------------------------------------------------------------
// Plan: the row streams
// ---------------------------------------------------------------------------------------

// Last column block of panel p (-1 for a panel without tiles).
__device__ __forceinline__ int64_t panel_last_cb(const int32_t* __restrict__ pt0, const int32_t* __restrict__ pnt,
                                                 const int32_t* __restrict__ tcol, int64_t p) {
  return pnt[p] > 0 ? (int64_t)tcol[pt0[p] + pnt[p] - 1] : -1;
}

// Thread per row: entries the row has in each panel of its row block.
__global__ void k_rs_counts(int64_t n, const int64_t* __restrict__ fptr, const int32_t* __restrict__ fcol,
                            const int32_t* __restrict__ rbp, const int32_t* __restrict__ pt0,
                            const int32_t* __restrict__ pnt, const int32_t* __restrict__ tcol,
                            uint16_t* __restrict__ cnt) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t I = r / kMR;
  const int lr = (int)(r - I * kMR);
  int64_t k = fptr[r];
  const int64_t kend = fptr[r + 1];
  for (int64_t p = rbp[I]; p < rbp[I + 1]; ++p) {
    const int64_t last = panel_last_cb(pt0, pnt, tcol, p);
    int c = 0;
    while (k < kend && (int64_t)(fcol[k] / kMC) <= last) {
      ++k;
      ++c;
    }
    cnt[p * kMR + lr] = (uint16_t)c;
  }
}

// CTA per panel: the panel's 256 rows ranked by entry count (descending, ties by row), so that
// each warp's 32 lanes take rows of near-equal length; steps of each warp = its longest row.
__global__ void __launch_bounds__(kMR) k_rs_rank(const uint16_t* __restrict__ cnt, uint8_t* __restrict__ perm,
                                                 int32_t* __restrict__ steps) {
  __shared__ uint16_t c[kMR];
  const int64_t p = blockIdx.x;
  const int t = threadIdx.x;
  c[t] = cnt[p * kMR + t];
  __syncthreads();
  const int mine = c[t];
  int rank = 0;
  for (int u = 0; u < kMR; ++u) {
    const int o = c[u];
    rank += (o > mine) || (o == mine && u < t);
  }
  perm[p * kMR + rank] = (uint8_t)t;
  if (rank % kRW == 0) steps[p * kW + rank / kRW] = mine;
}

// Every stream position starts as padding: value 0 and the zero row of the class its lane
// wants at that step.  Block layout: [lane][step], 32 lanes x 8 steps.
template <typename VS>
__global__ void k_rs_pads(int64_t nent, uint16_t* __restrict__ bcol, VS* __restrict__ bval) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nent) return;
  const int lane = (int)((e % kBE) / kBS), k = (int)(e % kBS);
  bcol[e] = (uint16_t)(kPR + ((lane + k) & 7));
  bval[e] = VS(0);
}

// Class (panel-local row mod 8) taken at a step whose lane wants class `want`: `want` while the
// row has entries of it, else one that keeps its class mod 4, then mod 2.  Lane l wants
// (l + step) mod 8, so the 8 lanes of a shared-memory phase read rows of 8 distinct classes.
// `nz`: bit c set while the row has entries of class c left.
__device__ __forceinline__ int pick_class(int want, unsigned nz) {
  const int order[8] = {0, 4, 2, 6, 1, 5, 3, 7};
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = want ^ order[t];
    if ((nz >> c) & 1u) return c;
  }
  return -1;
}

// Per-class counters held in registers: the 8 entries are only ever indexed by unrolled constant
// indices (a run-time index would move the array to local memory).
__device__ __forceinline__ int cls_get(const int (&a)[8], int c) {
  int v = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) v = (i == c) ? a[i] : v;
  return v;
}
__device__ __forceinline__ void cls_add(int (&a)[8], int c, int d) {
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] += (i == c) ? d : 0;
}
__device__ __forceinline__ int cls_take(int (&a)[8], int c) {  // a[c]++
  const int v = cls_get(a, c);
  cls_add(a, c, 1);
  return v;
}

// CTA per panel, thread per slot: the slot's row's entries of the panel, class-ordered (the
// diagonal entry last), into the lane's column of the warp's stream.  The row's segment is read
// in column order twice: once to count its entries per class, once to bucket their offsets by
// class (each bucket in column order) into `sc` at the segment's own positions in the mirrored
// CSR.  The class sequence is then chosen from the counts alone, and each streamed block's 8
// steps (panel-local columns and values, padding after the row's last entry) are assembled in
// registers and stored with 16-byte moves.  The tile of a column is looked up in the panel's
// tile list, staged in shared memory.  Launch: blockDim.x == kMR, one block per panel.
template <typename V>
__global__ void __launch_bounds__(kMR) k_rs_scatter(const int64_t* __restrict__ fptr, const int32_t* __restrict__ fcol,
                                                    const V* __restrict__ fval, int64_t n,
                                                    const int32_t* __restrict__ pan_rb, const int32_t* __restrict__ pt0,
                                                    const int32_t* __restrict__ pnt, const int32_t* __restrict__ tcol,
                                                    const uint8_t* __restrict__ perm, const int64_t* __restrict__ sboff,
                                                    uint16_t* __restrict__ sc, uint16_t* __restrict__ bcol,
                                                    V* __restrict__ bval) {
  static_assert(kBS == 8 && (kBS * sizeof(V)) % 16 == 0, "a lane's block is whole 16-byte pieces");
  __shared__ int32_t s_tc[kPT];
  const int64_t p = blockIdx.x;
  const int slot = threadIdx.x, w = slot / kRW, lane = slot % kRW;
  const int t0 = pt0[p], nt = pnt[p];
  if (slot < nt) s_tc[slot] = tcol[t0 + slot];
  __syncthreads();
  const int64_t r = (int64_t)pan_rb[p] * kMR + perm[p * kMR + slot];
  if (r >= n || nt == 0) return;
  // the row's entries in this panel: columns in the panel's tile range
  const int64_t first_cb = s_tc[0], last_cb = s_tc[nt - 1];
  int64_t e0 = fptr[r], e1 = fptr[r + 1];
  {
    int64_t lo = e0, hi = e1;
    while (lo < hi) {
      const int64_t m = (lo + hi) >> 1;
      if ((int64_t)(fcol[m] / kMC) < first_cb) lo = m + 1; else hi = m;
    }
    e0 = lo;
    hi = e1;
    while (lo < hi) {
      const int64_t m = (lo + hi) >> 1;
      if ((int64_t)(fcol[m] / kMC) <= last_cb) lo = m + 1; else hi = m;
    }
    e1 = lo;
  }
  const int len = (int)(e1 - e0);  // at most kPT * kMC
  // counts per class; the diagonal entry, if it lies in this panel, takes the row's last step:
  // the small off-diagonal terms are summed before the (typically much larger) diagonal one
  int left[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int ediag = -1;
  for (int q = 0; q < len; ++q) {
    const int32_t c = fcol[e0 + q];
    if ((int64_t)c == r) ediag = q;
    cls_add(left, c & 7, 1);
  }
  if (ediag >= 0) cls_add(left, fcol[e0 + ediag] & 7, -1);
  // class buckets: offsets into the segment, column order within a class
  int pos[8];
  unsigned nz = 0u;
  {
    int run = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      pos[c] = run;
      run += left[c];
      nz |= (left[c] > 0 ? 1u : 0u) << c;
    }
  }
  uint16_t* bucket = sc + e0;
  {
    int fill[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) fill[c] = pos[c];
    for (int q = 0; q < len; ++q) {
      if (q == ediag) continue;
      bucket[cls_take(fill, fcol[e0 + q] & 7)] = (uint16_t)q;
    }
  }
  // the steps, a streamed block (8 steps of this lane) at a time
  const int64_t blk0 = sboff[p * kW + w];
  for (int b = 0; b * kBS < len; ++b) {
    uint32_t cw[kBS / 2] = {0u, 0u, 0u, 0u};
    alignas(16) V vv[kBS];
#pragma unroll
    for (int j = 0; j < kBS; ++j) {
      const int k = b * kBS + j;
      uint32_t cc;
      V v;
      if (k < len) {
        int q;
        if (ediag >= 0 && k == len - 1) {
          q = ediag;
        } else {
          const int c = pick_class((lane + k) & 7, nz);
          q = bucket[cls_take(pos, c)];
          cls_add(left, c, -1);
          if (cls_get(left, c) == 0) nz &= ~(1u << c);
        }
        const int64_t e = e0 + q;
        const int32_t col = fcol[e];
        const int32_t J = col / kMC;
        int lo = 0, hi = nt - 1;  // position of J among the panel's tiles (ascending)
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_tc[mid] < J) lo = mid + 1; else hi = mid;
        }
        cc = (uint32_t)(lo * kMC + (col - J * kMC));
        v = fval[e];
      } else {  // padding, as k_rs_pads writes it
        cc = (uint32_t)(kPR + ((lane + k) & 7));
        v = V(0);
      }
      cw[j >> 1] |= cc << (16 * (j & 1));
      vv[j] = v;
    }
    const int64_t at = (blk0 + b) * kBE + lane * kBS;
    *reinterpret_cast<uint4*>(bcol + at) = make_uint4(cw[0], cw[1], cw[2], cw[3]);
    const uint4* src = reinterpret_cast<const uint4*>(vv);
    uint4* dst = reinterpret_cast<uint4*>(bval + at);
#pragma unroll
    for (int u = 0; u < (int)(kBS * sizeof(V) / 16); ++u) dst[u] = src[u];
  }
}

template <typename V>
eig_status rowstream_fill(SpmmPlan* P, const int32_t* tile_rb, const int32_t* tile_cb, int64_t n_up_tiles,
                          const int64_t* jt_ptr, const int32_t* jt_tile, cudaStream_t st) {
  const int64_t n = P->n;
  const int tb = 256;
  const int64_t gb = (n + tb - 1) / tb;
  const V* val = static_cast<const V*>(P->val);
  // 1. lower-part lengths and offsets of the mirrored CSR
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
  k_mir_upper<V><<<(unsigned)((n * 32 + tb - 1) / tb), tb, 0, st>>>(n, P->rowptr, P->col, val, lower.as<int64_t>(),
                                                                    fptr.as<int64_t>(), fcol.as<int32_t>(), fval.as<V>());
  EIG_LAUNCH_CHECK("k_mir_upper");
  cnt.release();
  off.release();
  lower.release();
  // 3. tiles of the mirrored matrix per row block, cut into panels of at most kPT tiles
  //    (balanced: a row block of t tiles takes ceil(t / kPT) panels of near-equal size; a row
  //    block without tiles still gets one empty panel so that its rows are written)
  DevBuf ftile_ptr, ftile_col;
  std::vector<int64_t> h_tptr;
  std::vector<int32_t> h_tcol;
  EIG_TRY(build_tile_lists(n, kMR, kMC, fptr.as<int64_t>(), fcol.as<int32_t>(), st, ftile_ptr, ftile_col, h_tptr,
                           h_tcol));
  const int64_t nRB = (n + kMR - 1) / kMR;
  std::vector<int32_t> rbp(nRB + 1, 0), pt0, pnt;
  for (int64_t I = 0; I < nRB; ++I) {
    const int64_t t0 = h_tptr[I], nt = h_tptr[I + 1] - t0;
    const int64_t np = std::max<int64_t>(1, (nt + kPT - 1) / kPT);
    int64_t t = t0;
    for (int64_t q = 0; q < np; ++q) {
      const int64_t sz = nt / np + (q < nt % np ? 1 : 0);
      pt0.push_back((int32_t)t);
      pnt.push_back((int32_t)sz);
      t += sz;
    }
    rbp[I + 1] = rbp[I] + (int32_t)np;
  }
  const int64_t npan = rbp[nRB];
  P->m_npan = npan;
  EIG_TRY(P->m_rbp.reserve((nRB + 1) * 4));
  EIG_TRY(P->m_pt0.reserve(npan * 4));
  EIG_TRY(P->m_pnt.reserve(npan * 4));
  EIG_TRY(P->m_tcol.reserve(std::max<size_t>(h_tcol.size(), 1) * 4));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->m_rbp.p, rbp.data(), (nRB + 1) * 4, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->m_pt0.p, pt0.data(), npan * 4, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->m_pnt.p, pnt.data(), npan * 4, cudaMemcpyHostToDevice, st));
  if (!h_tcol.empty())
    EIG_CUDA_TRY(cudaMemcpyAsync(P->m_tcol.p, h_tcol.data(), h_tcol.size() * 4, cudaMemcpyHostToDevice, st));
  ftile_ptr.release();
  ftile_col.release();
  // 4. entries per (panel, row); rows ranked per panel; steps per (panel, warp); stream offsets
  std::vector<int32_t> pan_rb(npan);
  for (int64_t I = 0; I < nRB; ++I)
    for (int32_t q = rbp[I]; q < rbp[I + 1]; ++q) pan_rb[q] = (int32_t)I;
  DevBuf d_pan_rb, cntp, steps;
  EIG_TRY(d_pan_rb.reserve(npan * 4));
  EIG_CUDA_TRY(cudaMemcpyAsync(d_pan_rb.p, pan_rb.data(), npan * 4, cudaMemcpyHostToDevice, st));
  EIG_TRY(cntp.reserve(npan * kMR * 2));
  EIG_CUDA_TRY(cudaMemsetAsync(cntp.p, 0, npan * kMR * 2, st));
  k_rs_counts<<<(unsigned)gb, tb, 0, st>>>(n, fptr.as<int64_t>(), fcol.as<int32_t>(), P->m_rbp.as<int32_t>(),
                                           P->m_pt0.as<int32_t>(), P->m_pnt.as<int32_t>(), P->m_tcol.as<int32_t>(),
                                           cntp.as<uint16_t>());
  EIG_LAUNCH_CHECK("k_rs_counts");
  EIG_TRY(P->m_perm.reserve(npan * kMR));
  EIG_TRY(steps.reserve(npan * kW * 4));
  k_rs_rank<<<(unsigned)npan, kMR, 0, st>>>(cntp.as<uint16_t>(), P->m_perm.as<uint8_t>(), steps.as<int32_t>());
  EIG_LAUNCH_CHECK("k_rs_rank");
  std::vector<int32_t> h_steps(npan * kW);
  std::vector<int64_t> sboff(npan * kW + 1, 0);
  EIG_CUDA_TRY(cudaMemcpyAsync(h_steps.data(), steps.p, npan * kW * 4, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t i = 0; i < npan * kW; ++i) sboff[i + 1] = sboff[i] + (h_steps[i] + kBS - 1) / kBS;
  const int64_t nblk = sboff[npan * kW];
  P->m_nblk = nblk;
  EIG_TRY(P->m_steps.reserve(npan * kW * 4));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->m_steps.p, steps.p, npan * kW * 4, cudaMemcpyDeviceToDevice, st));
  EIG_TRY(P->m_sboff.reserve((npan * kW + 1) * 8));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->m_sboff.p, sboff.data(), (npan * kW + 1) * 8, cudaMemcpyHostToDevice, st));
  // 5. the streams: padding everywhere, then each row's entries into its lane
  const int64_t nent = std::max<int64_t>(nblk, 1) * kBE;
  EIG_TRY(P->m_bcol.reserve(nent * 2));
  EIG_TRY(P->m_bval.reserve(nent * sizeof(V)));
  k_rs_pads<V><<<(unsigned)((nent + tb - 1) / tb), tb, 0, st>>>(nent, P->m_bcol.as<uint16_t>(), P->m_bval.as<V>());
  EIG_LAUNCH_CHECK("k_rs_pads");
  if (npan > 0) {
    DevBuf sc;  // class buckets, at each row segment's positions in the mirrored CSR
    EIG_TRY(sc.reserve(std::max<int64_t>(fnnz, 1) * 2));
    k_rs_scatter<V><<<(unsigned)npan, kMR, 0, st>>>(
        fptr.as<int64_t>(), fcol.as<int32_t>(), fval.as<V>(), n, d_pan_rb.as<int32_t>(), P->m_pt0.as<int32_t>(),
        P->m_pnt.as<int32_t>(), P->m_tcol.as<int32_t>(), P->m_perm.as<uint8_t>(), P->m_sboff.as<int64_t>(),
        sc.as<uint16_t>(), P->m_bcol.as<uint16_t>(), P->m_bval.as<V>());
    EIG_LAUNCH_CHECK("k_rs_scatter");
  }
  EIG_CUDA_TRY(cudaStreamSynchronize(st));  // temporaries go out of scope
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------------------
struct RsArgs {
  int64_t n;
  const int32_t* rbp;
  const int32_t* pt0;
  const int32_t* pnt;
  const int32_t* tcol;
  const uint8_t* perm;
  const int32_t* steps;
  const int64_t* sboff;
  const uint16_t* bcol;
  const void* bval;
  int* err;
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

// One product of a batched launch, and the batch (passed by value: at most kBatchJobs jobs).
struct MirrorJob {
  RsArgs a;
  const void* X;
  void* Y;
  int ld, col0, xj_bulk;
  MirrorEpi epi;
};
constexpr int kBatchJobs = 64;
struct MirrorBatch {
  int n;
  int64_t cta0[kBatchJobs + 1];
  MirrorJob jobs[kBatchJobs];
};

// Double-float accumulation applies to FP64 vectors with FP32 or BF16 values.
template <typename T, typename V> struct MirrorDF { static constexpr bool value = false; };
template <> struct MirrorDF<double, float> { static constexpr bool value = true; };
template <> struct MirrorDF<double, uint16_t> { static constexpr bool value = true; };

// Lane geometry for (vector type T, value type V, kernel block width NB).
//   ES: bytes of one staged X element (FP32; FP64; or a (hi, lo) FP32 pair for double-float);
//   RBY: bytes of one staged X row, gathered by each lane as NCH pieces of LDB bytes.
template <typename T, typename V, int NB> struct RsShape {
  static constexpr bool DF = MirrorDF<T, V>::value;
  static constexpr int ES = (int)sizeof(T);
  static constexpr int RBY = NB * ES;
  static constexpr int LDB = RBY >= 16 ? 16 : RBY;
  static constexpr int NCH = RBY / LDB;       // pieces per row
  static constexpr int EPC = LDB / ES;        // elements per piece
  // lanes of a phase reading the same bank-line offset class get distinct pieces
  static constexpr int ROTDIV = NCH >= 8 ? 1 : 8 / NCH;
  static constexpr size_t XBYTES = (size_t)(kPR + 8) * RBY;
  static constexpr int MINB0 = (int)(233472 / (XBYTES + 1024 + 128));
  // register budget: up to 4 CTAs per SM for rows of <= 16 bytes, 3 for 32, else (and for
  // FP64 values, whose blocks take twice the registers) 2
  static constexpr int MAXB = sizeof(typename ValLoad<V>::storage) == 8 ? 2 : (RBY <= 16 ? 4 : (RBY <= 32 ? 3 : 2));
  static constexpr int MINB = MINB0 < 1 ? 1 : (MINB0 > MAXB ? MAXB : MINB0);   // resident CTAs per SM
  // streamed blocks held in registers: the next block loads while the current one runs
  static constexpr int PF = 2;
  static constexpr int VW = (kBS * (int)sizeof(typename ValLoad<V>::storage)) / 4;   // value words per block
};

// Streamed loads: bypass L1, evict first from L2 (each entry is read once per product).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint4 ldg_stream(const void* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
// Bulk prefetch of a global range into L2 (no registers, no shared memory).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                 uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// Shared-memory piece loads of 4, 8 or 16 bytes (raw words).
template <int B> struct SLd;
template <> struct SLd<4> {
  __device__ __forceinline__ static void ld(uint32_t a, uint32_t* w) {
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w[0]) : "r"(a));
  }
};
template <> struct SLd<8> {
  __device__ __forceinline__ static void ld(uint32_t a, uint32_t* w) {
    asm volatile("ld.shared.v2.b32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "r"(a));
  }
};
template <> struct SLd<16> {
  __device__ __forceinline__ static void ld(uint32_t a, uint32_t* w) {
    asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "r"(a));
  }
};

// y += v * x over a lane's N elements, x given as raw staged words.
template <typename T, int N, bool DF> struct RsAcc;
template <int N> struct RsAcc<float, N, false> {
  typedef float VT;
  typedef float OT;
  static constexpr int N2 = (N + 1) / 2;
  float2 y[N2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int e = 0; e < N2; ++e) y[e] = make_float2(0.0f, 0.0f);
  }
  __device__ __forceinline__ void add(int slot0, float v, const uint32_t* w, int nw) {
    if (nw % 2 == 0) {
      // packed FP32x2 multiply-add (sm_100+): two elements of y per instruction
      const float2 vv = make_float2(v, v);
#pragma unroll
      for (int e = 0; e < nw; e += 2) {
        const int s = (slot0 + e) / 2;
        y[s] = __ffma2_rn(vv, make_float2(__uint_as_float(w[e]), __uint_as_float(w[e + 1])), y[s]);
      }
    } else {
      y[slot0 / 2].x = fmaf(v, __uint_as_float(w[0]), y[slot0 / 2].x);
    }
  }
  __device__ __forceinline__ OT get(int e) const { return (e & 1) ? y[e / 2].y : y[e / 2].x; }
};
template <int N> struct RsAcc<double, N, false> {
  typedef double VT;
  typedef double OT;
  double y[N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int e = 0; e < N; ++e) y[e] = 0.0;
  }
  __device__ __forceinline__ void add(int slot0, double v, const uint32_t* w, int nw) {
#pragma unroll
    for (int e = 0; e < nw / 2; ++e) y[slot0 + e] = fma(v, __hiloint2double(w[2 * e + 1], w[2 * e]), y[slot0 + e]);
  }
  __device__ __forceinline__ OT get(int e) const { return y[e]; }
};
// Double-float: X staged as (hi, lo) FP32 pairs (8 bytes per element, like FP64); each product
// v * hi taken exactly (FMA two-product), summed into hi by two-sum, every error term and v * lo
// into lo: ~2^-44 relative per step, at FP32 instruction rate.  A 16-byte piece holds two
// elements as (hi_e, hi_e+1, lo_e, lo_e+1), so a step is FP32x2 arithmetic on element pairs;
// every operation is an explicit round-to-nearest (a subtraction b - a is fma(a, -1, b)), so no
// contraction can break the two-sum.  A one-element piece (block width 1) holds (hi, lo).
template <int N> struct RsAcc<double, N, true> {
  typedef float VT;
  typedef double OT;
  static constexpr int N2 = (N + 1) / 2;
  float2 hi[N2], lo[N2];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int e = 0; e < N2; ++e) hi[e] = lo[e] = make_float2(0.0f, 0.0f);
  }
  __device__ __forceinline__ void add(int slot0, float v, const uint32_t* w, int nw) {
    if (nw == 4) {
      const int s = slot0 / 2;
      const float2 vv = make_float2(v, v), nv = make_float2(-v, -v), m1 = make_float2(-1.0f, -1.0f);
      const float2 xh = make_float2(__uint_as_float(w[0]), __uint_as_float(w[1]));
      const float2 xl = make_float2(__uint_as_float(w[2]), __uint_as_float(w[3]));
      const float2 p = __fmul2_rn(vv, xh);
      const float2 q = __ffma2_rn(nv, xh, p);                          // p - v hi: minus the product's error
      const float2 t = __fadd2_rn(hi[s], p);
      const float2 bb = __ffma2_rn(hi[s], m1, t);                      // t - hi
      const float2 e1 = __ffma2_rn(__ffma2_rn(bb, m1, t), m1, hi[s]);  // hi - (t - bb)
      const float2 e2 = __ffma2_rn(bb, m1, p);                         // p - bb
      const float2 err = __fadd2_rn(e1, e2);
      hi[s] = t;
      lo[s] = __ffma2_rn(vv, xl, __fadd2_rn(lo[s], __ffma2_rn(q, m1, err)));
    } else {
      float& h = (slot0 & 1) ? hi[slot0 / 2].y : hi[slot0 / 2].x;
      float& l = (slot0 & 1) ? lo[slot0 / 2].y : lo[slot0 / 2].x;
      const float xh = __uint_as_float(w[0]), xl = __uint_as_float(w[1]);
      const float p = __fmul_rn(v, xh);
      const float pe = __fmaf_rn(v, xh, -p);
      const float t = __fadd_rn(h, p);
      const float bb = __fsub_rn(t, h);
      const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bb)), __fsub_rn(p, bb));
      h = t;
      l = __fmaf_rn(v, xl, __fadd_rn(l, __fadd_rn(err, pe)));
    }
  }
  __device__ __forceinline__ OT get(int e) const {
    return (e & 1) ? (double)hi[e / 2].y + (double)lo[e / 2].y : (double)hi[e / 2].x + (double)lo[e / 2].x;
  }
};

// Value k (0..7) of a lane's streamed block, widened to the arithmetic type.
template <typename VS, typename VT> struct BlkVal;
template <typename VT> struct BlkVal<float, VT> {
  __device__ __forceinline__ static VT get(const uint32_t* w, int i) { return (VT)__uint_as_float(w[i]); }
};
template <typename VT> struct BlkVal<uint16_t, VT> {
  __device__ __forceinline__ static VT get(const uint32_t* w, int i) {
    const uint32_t u = w[i >> 1];
    return (VT)__uint_as_float((i & 1) ? (u & 0xFFFF0000u) : (u << 16));
  }
};
template <typename VT> struct BlkVal<double, VT> {
  __device__ __forceinline__ static VT get(const uint32_t* w, int i) {
    return (VT)__hiloint2double(w[2 * i + 1], w[2 * i]);
  }
};

// One staged X element of type T (FP32, FP64; double-float pairs are staged from FP64).
template <typename T, bool DF> struct Stage;
template <> struct Stage<float, false> {
  __device__ __forceinline__ static void put(unsigned char* row, int e, int, float x) {
    reinterpret_cast<float*>(row)[e] = x;
  }
};
template <> struct Stage<double, false> {
  __device__ __forceinline__ static void put(unsigned char* row, int e, int, double x) {
    reinterpret_cast<double*>(row)[e] = x;
  }
};
template <> struct Stage<double, true> {
  // element e of a staged row: hi and lo words in the piece layout of the double-float
  // accumulator (pairs of elements per 16-byte piece, or (hi, lo) for one-element rows)
  __device__ __forceinline__ static void put(unsigned char* row, int e, int nb, double x) {
    const float h = __double2float_rn(x);
    float* d = reinterpret_cast<float*>(row);
    const int ih = nb == 1 ? 0 : (e >> 1) * 4 + (e & 1);
    const int il = nb == 1 ? 1 : ih + 2;
    d[ih] = h;
    d[il] = __double2float_rn(x - (double)h);
  }
};

// Row block I of one product.  Y (and X, Qp) rows have stride ld elements; the product covers
// elements [col0, col0 + NB).
template <typename T, typename V, int NB, bool CHEB>
__device__ __forceinline__ void mirror_row_block(const RsArgs& a, const T* __restrict__ X, T* __restrict__ Y, int ld,
                                                 int col0, int xj_bulk, const MirrorEpi& epi, int64_t I) {
  typedef RsShape<T, V, NB> Sh;
  constexpr bool DF = Sh::DF;
  constexpr int RBY = Sh::RBY, LDB = Sh::LDB, NCH = Sh::NCH, EPC = Sh::EPC, PF = Sh::PF, VW = Sh::VW;
  constexpr int NW = LDB / 4;  // words per piece
  typedef typename ValLoad<V>::storage VS;
  typedef RsAcc<T, NB, DF> Acc;
  typedef typename Acc::VT VT;
  typedef typename Acc::OT OT;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* xs = smem;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sh::XBYTES);
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t r0 = I * kMR;
  const int p0 = a.rbp[I], p1 = a.rbp[I + 1];

  // zero rows (one per class) for the padding entries; never overwritten by staging
  for (int i = tid; i < 8 * RBY / 4; i += kW * 32) reinterpret_cast<uint32_t*>(xs + (size_t)kPR * RBY)[i] = 0u;
  if (tid == 0) {
    s_abort = 0;
    mbar_init(bar, 1);
    mbar_init_fence();
  }
  // this lane's pieces start at piece `rot` of the row (distinct among the lanes of a phase
  // whose rows share a bank-line offset)
  const int rot = (lane / Sh::ROTDIV) % NCH;
  uint32_t poff[NCH];
#pragma unroll
  for (int j = 0; j < NCH; ++j) poff[j] = (uint32_t)(((j + rot) % NCH) * LDB);
  const uint32_t xs_a = smem_u32(xs);
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const uint16_t* bcol = a.bcol;
  const VS* bval = static_cast<const VS*>(a.bval);
  uint32_t xphase = 0;

  for (int p = p0; p < p1; ++p) {
    __syncthreads();  // the previous panel's gathers are done
    const int t0 = a.pt0[p], npt = a.pnt[p];
    if (xj_bulk) {
      if (tid == 0 && npt > 0) {
        uint32_t tot = 0;
        for (int t = 0; t < npt; ++t) {
          const int64_t cb0 = (int64_t)a.tcol[t0 + t] * kMC;
          tot += (uint32_t)(min64(kMC, a.n - cb0) * RBY);
        }
        mbar_arrive_expect_tx(bar, tot);
        for (int t = 0; t < npt; ++t) {
          const int64_t cb0 = (int64_t)a.tcol[t0 + t] * kMC;
          const uint32_t bytes = (uint32_t)(min64(kMC, a.n - cb0) * RBY);
          tma_load_1d_hint(xs + (size_t)t * kMC * RBY, X + cb0 * NB, bytes, bar, pol_keep);
        }
      }
      if (npt > 0) {
        if (!mbar_wait_bounded(bar, xphase)) {
          atomicOr(a.err, 1);
          s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        xphase ^= 1u;
      }
    } else {
      for (int64_t i = tid; i < (int64_t)npt * kMC * NB; i += kW * 32) {
        const int t = (int)(i / (kMC * NB));
        const int rr = (int)((i / NB) % kMC), e = (int)(i % NB);
        const int64_t row = (int64_t)a.tcol[t0 + t] * kMC + rr;
        if (row < a.n) Stage<T, DF>::put(xs + (size_t)(t * kMC + rr) * RBY, e, NB, X[row * ld + col0 + e]);
      }
      __syncthreads();
    }

    // this lane's row and the warp's stream
    const int64_t r = r0 + a.perm[(int64_t)p * kMR + w * 32 + lane];
    const int L = a.steps[(int64_t)p * kW + w];
    const int64_t b0 = a.sboff[(int64_t)p * kW + w];
    const int nb = (L + kBS - 1) / kBS;
    Acc acc;
    acc.zero();
    uint4 bc[PF];
    uint32_t bv[PF][VW];
    auto load_blk = [&](int b, int s) {
      const int64_t e = (b0 + b) * kBE + lane * kBS;
      bc[s] = ldg_stream(bcol + e, pol_stream);
#pragma unroll
      for (int u = 0; u < VW; u += 4) {
        const uint4 t = ldg_stream(reinterpret_cast<const unsigned char*>(bval + e) + u * 4, pol_stream);
        bv[s][u] = t.x; bv[s][u + 1] = t.y; bv[s][u + 2] = t.z; bv[s][u + 3] = t.w;
      }
    };
    // blocks kL2 ahead of the one running are prefetched into L2 by lane 0, so that the
    // register loads one block ahead see L2 rather than HBM latency
    auto prefetch_blk = [&](int b) {
      if (lane == 0 && b < nb) {
        prefetch_l2(bcol + (b0 + b) * kBE, kBE * 2);
        prefetch_l2(bval + (b0 + b) * kBE, kBE * (uint32_t)sizeof(VS));
      }
    };
    for (int b = 0; b < kL2; ++b) prefetch_blk(b);
#pragma unroll
    for (int s = 0; s < PF; ++s)
      if (s < nb) load_blk(s, s);
    for (int b = 0; b < nb; b += PF) {
#pragma unroll
      for (int s = 0; s < PF; ++s) {
        if (b + s < nb) {
          prefetch_blk(b + s + kL2);
          const uint32_t cw[4] = {bc[s].x, bc[s].y, bc[s].z, bc[s].w};
          uint32_t vw[VW];
#pragma unroll
          for (int u = 0; u < VW; ++u) vw[u] = bv[s][u];
          if (b + s + PF < nb) load_blk(b + s + PF, s);
          const int ks = min(kBS, L - (b + s) * kBS);   // steps in this block (warp-uniform)
          auto step = [&](int k) {
            const uint32_t c = (k & 1) ? (cw[k >> 1] >> 16) : (cw[k >> 1] & 0xFFFFu);
            const VT v = BlkVal<VS, VT>::get(vw, k);
            const uint32_t rowa = xs_a + c * (uint32_t)RBY;
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
              uint32_t xw[NW];
              SLd<LDB>::ld(rowa + poff[j], xw);
              acc.add(j * EPC, v, xw, NW);
            }
          };
          if (ks == kBS) {
            // a whole block: straight-line code, so the gathers of later steps can be issued
            // ahead of the multiply-adds of earlier ones
#pragma unroll
            for (int k = 0; k < kBS; ++k) step(k);
          } else {
#pragma unroll
            for (int k = 0; k < kBS; ++k)
              if (k < ks) step(k);
          }
        }
      }
    }
    // the row's sum over this panel: stored (first panel) or added to the earlier panels'
    if (r < a.n) {
      const bool first_panel = (p == p0), last_panel = (p == p1 - 1);
#pragma unroll
      for (int j = 0; j < NCH; ++j) {
        const int jc0 = col0 + ((j + rot) % NCH) * EPC;   // first element of the piece
        T* yp = Y + r * ld + jc0;
        OT v[EPC];
#pragma unroll
        for (int e = 0; e < EPC; ++e) v[e] = acc.get(j * EPC + e);
        if (!first_panel) {
          const Vec<T, EPC> old = VecIO<T, EPC>::ld(yp);
#pragma unroll
          for (int e = 0; e < EPC; ++e) v[e] += (OT)old.v[e];
        }
        Vec<T, EPC> out;
        if (CHEB && last_panel) {
          const Vec<T, EPC> xv = VecIO<T, EPC>::ld(X + r * ld + jc0);
          Vec<T, EPC> qv;
          qv.zero();
          if (!epi.first) qv = VecIO<T, EPC>::ld(static_cast<const T*>(epi.Qp) + r * ld + jc0);
#pragma unroll
          for (int e = 0; e < EPC; ++e) {
            if (!epi.active[jc0 + e]) {
              out.v[e] = xv.v[e];
            } else {
              // explicit roundings, as the separate elementwise step (k_cheb) takes them: the
              // single and the batched launch then agree bit for bit
              double yv = __dmul_rn(epi.a, __fma_rn(-epi.c, (double)xv.v[e], (double)(T)v[e]));
              if (!epi.first) yv = __dsub_rn(yv, (double)qv.v[e]);
              out.v[e] = (T)yv;
            }
          }
        } else {
#pragma unroll
          for (int e = 0; e < EPC; ++e) out.v[e] = (T)v[e];
        }
        VecIO<T, EPC>::st(yp, out);
      }
    }
  }
  if (s_abort) {
    // leave no bulk copy in flight into this CTA's shared memory (bounded wait on the phase
    // that gave up)
    if (tid == 0) (void)mbar_wait_bounded(bar, xphase);
    __syncthreads();
  }
}

// One product: CTA = row block.
template <typename T, typename V, int NB, bool CHEB>
__global__ void __launch_bounds__(kW * 32, RsShape<T, V, NB>::MINB)
k_spmm_mirror(const __grid_constant__ RsArgs a, const T* __restrict__ X, T* __restrict__ Y, int ld, int col0,
              int xj_bulk, const __grid_constant__ MirrorEpi epi) {
  mirror_row_block<T, V, NB, CHEB>(a, X, Y, ld, col0, xj_bulk, epi, blockIdx.x);
}

// Several products of one shape in one launch over their concatenated row blocks (the
// (instance, row block) work list of a batch): job j owns CTAs [cta0[j], cta0[j + 1]).
template <typename T, typename V, int NB, bool CHEB>
__global__ void __launch_bounds__(kW * 32, RsShape<T, V, NB>::MINB)
k_spmm_mirror_batch(const __grid_constant__ MirrorBatch B) {
  int j = 0;
  while (j + 1 < B.n && B.cta0[j + 1] <= (int64_t)blockIdx.x) ++j;
  const MirrorJob& J = B.jobs[j];
  mirror_row_block<T, V, NB, CHEB>(J.a, static_cast<const T*>(J.X), static_cast<T*>(J.Y), J.ld, J.col0, J.xj_bulk,
                                   J.epi, (int64_t)blockIdx.x - B.cta0[j]);
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
size_t mirror_bytes_estimate(const SpmmPlan* P) {
  // mirrored CSR (temporary) + streams of 2-byte columns and values with ~5% padding
  const double fnnz = 2.0 * double(P->nnz);
  const double vb = double(dtype_size(P->val_type));
  return (size_t)(fnnz * (4.0 + vb) + 1.1 * fnnz * (2.0 + vb) + 64.0 * double(P->n));
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
  eig_status s;
  if (P->val_type == EIG_F32)
    s = rowstream_fill<float>(P, d_trb.as<int32_t>(), d_tcb.as<int32_t>(), nt, d_jptr.as<int64_t>(),
                              d_jt.as<int32_t>(), st);
  else if (P->val_type == EIG_F64)
    s = rowstream_fill<double>(P, d_trb.as<int32_t>(), d_tcb.as<int32_t>(), nt, d_jptr.as<int64_t>(),
                               d_jt.as<int32_t>(), st);
  else
    s = rowstream_fill<uint16_t>(P, d_trb.as<int32_t>(), d_tcb.as<int32_t>(), nt, d_jptr.as<int64_t>(),
                                 d_jt.as<int32_t>(), st);
  EIG_TRY(s);
  if (!P->err.p) {
    EIG_TRY(P->err.reserve(16));
    EIG_CUDA_TRY(cudaMemsetAsync(P->err.p, 0, 16, st));
    EIG_CUDA_TRY(cudaStreamSynchronize(st));
  }
  P->mirrored = true;
  return EIG_OK;
}

// Kernel block width for (T, V, NB): NB itself while one panel of staged X rows fits in a
// CTA's shared memory, else a column slice of it (the product then runs as several launches
// over column slices, each reading the matrix once).
template <typename T, typename V, int NB> struct RsSlice {
  static constexpr int value =
      (RsShape<T, V, NB>::XBYTES + 1024 <= 232448 || NB == 1) ? NB : RsSlice<T, V, NB / 2>::value;
};
template <typename T, typename V> struct RsSlice<T, V, 1> { static constexpr int value = 1; };

// The plan's row streams as kernel arguments.
static RsArgs rs_args(SpmmPlan* P) {
  RsArgs a;
  a.n = P->n;
  a.rbp = P->m_rbp.as<int32_t>();
  a.pt0 = P->m_pt0.as<int32_t>();
  a.pnt = P->m_pnt.as<int32_t>();
  a.tcol = P->m_tcol.as<int32_t>();
  a.perm = P->m_perm.as<uint8_t>();
  a.steps = P->m_steps.as<int32_t>();
  a.sboff = P->m_sboff.as<int64_t>();
  a.bcol = P->m_bcol.as<uint16_t>();
  a.bval = P->m_bval.p;
  a.err = P->err.as<int>();
  return a;
}

// X tiles by bulk copy: plain staging of whole, 16-byte aligned rows of a 16-byte multiple.
template <typename T, typename V, int NBK>
static int rs_xj_bulk(const T* X, int ld) {
  typedef RsShape<T, V, NBK> Sh;
  return !Sh::DF && ld == NBK && (Sh::RBY % 16 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15u) == 0);
}

template <typename T, typename V, int NBK, bool CHEB>
static eig_status rs_launch(SpmmPlan* P, const T* X, T* Y, int ld, int col0, const MirrorEpi& epi, cudaStream_t st) {
  typedef RsShape<T, V, NBK> Sh;
  int dev = 0, maxsm = 0;
  EIG_CUDA_TRY(cudaGetDevice(&dev));
  EIG_CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t sm = Sh::XBYTES + 16;
  if (sm > (size_t)maxsm) return EIG_EUNSUPPORTED;
  const RsArgs a = rs_args(P);
  const int xj_bulk = rs_xj_bulk<T, V, NBK>(X, ld);
  auto kern = k_spmm_mirror<T, V, NBK, CHEB>;
  EIG_CUDA_TRY(::eig::ensure_dyn_smem(kern, (int)sm));
  kern<<<(unsigned)P->nRB, kW * 32, sm, st>>>(a, X, Y, ld, col0, xj_bulk, epi);
  EIG_LAUNCH_CHECK(CHEB ? "k_spmm_mirror_cheb" : "k_spmm_mirror");
  return EIG_OK;
}

template <typename T, typename V, int NB>
eig_status mirror_launch(SpmmPlan* P, const T* X, T* Y, cudaStream_t st) {
  constexpr int NBK = RsSlice<T, V, NB>::value;
  for (int c0 = 0; c0 < NB; c0 += NBK) EIG_TRY((rs_launch<T, V, NBK, false>(P, X, Y, NB, c0, MirrorEpi(), st)));
  return EIG_OK;
}

// Several products of one shape, each Y_i = H_i X_i (CHEB: the fused Chebyshev step with its
// own Qp_i, active_i, alpha_i, c_i), in one launch per at most kBatchJobs column slices over
// their concatenated row blocks; the sums are those of the single launch.
template <typename T, typename V, int NB, bool CHEB>
eig_status mirror_launch_batch(const SpmmJob* jobs, int count, cudaStream_t st) {
  constexpr int NBK = RsSlice<T, V, NB>::value;
  typedef RsShape<T, V, NBK> Sh;
  int dev = 0, maxsm = 0;
  EIG_CUDA_TRY(cudaGetDevice(&dev));
  EIG_CUDA_TRY(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t sm = Sh::XBYTES + 16;
  if (sm > (size_t)maxsm) return EIG_EUNSUPPORTED;
  for (int i = 0; i < count; ++i)
    if (!jobs[i].P->mirrored) return EIG_EUNSUPPORTED;
  auto kern = k_spmm_mirror_batch<T, V, NBK, CHEB>;
  EIG_CUDA_TRY(::eig::ensure_dyn_smem(kern, (int)sm));
  MirrorBatch B;
  B.n = 0;
  int64_t ctas = 0;
  auto flush = [&]() -> eig_status {
    if (B.n == 0) return EIG_OK;
    B.cta0[B.n] = ctas;
    kern<<<(unsigned)ctas, kW * 32, sm, st>>>(B);
    EIG_LAUNCH_CHECK(CHEB ? "k_spmm_mirror_batch_cheb" : "k_spmm_mirror_batch");
    B.n = 0;
    ctas = 0;
    return EIG_OK;
  };
  for (int i = 0; i < count; ++i) {
    const SpmmJob& q = jobs[i];
    for (int c0 = 0; c0 < NB; c0 += NBK) {
      MirrorJob& J = B.jobs[B.n];
      J.a = rs_args(q.P);
      J.X = q.X;
      J.Y = q.Y;
      J.ld = NB;
      J.col0 = c0;
      J.xj_bulk = rs_xj_bulk<T, V, NBK>(static_cast<const T*>(q.X), NB);
      J.epi = MirrorEpi();
      if (CHEB) {
        J.epi.Qp = q.Qp;
        J.epi.active = q.active;
        J.epi.a = q.alpha;
        J.epi.c = q.c;
        J.epi.first = q.first;
      }
      B.cta0[B.n] = ctas;
      ctas += q.P->nRB;
      if (++B.n == kBatchJobs) EIG_TRY(flush());
    }
  }
  return flush();
}

#define EIG_MIRROR_BATCH_INST(T, V)                                                                    \
  template eig_status mirror_launch_batch<T, V, 8, false>(const SpmmJob*, int, cudaStream_t);           \
  template eig_status mirror_launch_batch<T, V, 16, false>(const SpmmJob*, int, cudaStream_t);          \
  template eig_status mirror_launch_batch<T, V, 8, true>(const SpmmJob*, int, cudaStream_t);            \
  template eig_status mirror_launch_batch<T, V, 16, true>(const SpmmJob*, int, cudaStream_t);
EIG_MIRROR_BATCH_INST(float, float)
EIG_MIRROR_BATCH_INST(double, float)

// One column of X (row stride ld, column col) times H into the same column of Y: the SpMV of
// a decoupled RMM-DIIS vector (Sec. 4.3), summed in the order of the block product's column.
template <typename T, typename V>
eig_status mirror_launch_column(SpmmPlan* P, const T* X, T* Y, int ld, int col, cudaStream_t st) {
  return rs_launch<T, V, 1, false>(P, X, Y, ld, col, MirrorEpi(), st);
}

// The Chebyshev-step variant (same kernel, fused epilogue).
template <typename T, typename V, int NB>
eig_status mirror_launch_cheb(SpmmPlan* P, const T* X, T* Y, const T* Qp, const int* active, double alpha, double c,
                              int first, cudaStream_t st) {
  MirrorEpi epi;
  epi.Qp = Qp;
  epi.active = active;
  epi.a = alpha;
  epi.c = c;
  epi.first = first;
  constexpr int NBK = RsSlice<T, V, NB>::value;
  for (int c0 = 0; c0 < NB; c0 += NBK) EIG_TRY((rs_launch<T, V, NBK, true>(P, X, Y, NB, c0, epi, st)));
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

template eig_status mirror_launch_column<float, float>(SpmmPlan*, const float*, float*, int, int, cudaStream_t);
template eig_status mirror_launch_column<float, uint16_t>(SpmmPlan*, const float*, float*, int, int, cudaStream_t);
template eig_status mirror_launch_column<double, double>(SpmmPlan*, const double*, double*, int, int, cudaStream_t);
template eig_status mirror_launch_column<double, float>(SpmmPlan*, const double*, double*, int, int, cudaStream_t);
template eig_status mirror_launch_column<double, uint16_t>(SpmmPlan*, const double*, double*, int, int,
                                                           cudaStream_t);

}  // namespace eig
