// Symmetric half-stored block SpMM, Y = H X with H = U + U_strict^T (Sec. 1; Eqs. upd1-upd2;
// Sec. 3.1 stores only half of H).
//
// Design (GB300-first):
//   * rows are grouped in row blocks of R rows; one CTA owns a row block, columns are cut in
//     column blocks of C; a nonempty (row block, column block) pair is a tile;
//   * per tile the CTA stages X_J (C x nb) in shared memory, every warp walks its rows'
//     entries in that column block (a row's entries are contiguous there because CSR rows
//     are sorted) and does, per entry (r, c, v):
//        y_r += v * X_J[c]        (gather, accumulated in registers across the entries)
//        z_c += v * X_I[r]        (transposed half, into the warp's private z in smem)
//     with lanes laid out as (entry, 16-byte slice of the nb-wide row), so shared memory
//     traffic is 128-bit;
//   * the warps' private z are summed in a fixed order: for a tile inside the CTA's own row
//     range the sum is added to the CTA's y, otherwise it is written to a scratch slot;
//   * a second kernel adds the scratch slots into Y following the transpose schedule
//     (slots of each column block in ascending source-row-block order).
//   No atomics touch floating-point data, so Y is bitwise reproducible.
#include "common.cuh"
#include "spmm.cuh"
#include "vec.cuh"

#include <algorithm>

namespace eig {

// ---------------------------------------------------------------------------------------
// Plan construction kernels
// ---------------------------------------------------------------------------------------
__global__ void k_validate_csr(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               int64_t nnz, int* __restrict__ bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t a = rowptr[i], b = rowptr[i + 1];
  if (a > b || a < 0 || b > nnz) { atomicOr(bad, 1); return; }
  int64_t prev = i - 1;
  for (int64_t k = a; k < b; ++k) {
    int64_t c = col[k];
    if (c <= prev || c >= n) { atomicOr(bad, 2); return; }
    prev = c;
  }
}

__global__ void k_extract_diag(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const void* __restrict__ val, int vt, double* __restrict__ diag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t a = rowptr[i], b = rowptr[i + 1];
  double d = 0.0;
  if (a < b && col[a] == i) {
    if (vt == EIG_F64) d = static_cast<const double*>(val)[a];
    else if (vt == EIG_F32) d = static_cast<const float*>(val)[a];
    else d = bf16_to_f32(static_cast<const uint16_t*>(val)[a]);
  }
  diag[i] = d;
}

// One thread per row: mark the column blocks its entries touch in the (row block x column
// block) bitmap.  atomicOr on integer words only: the bitmap is order independent.
__global__ void k_tile_bitmap(int64_t n, int R, int C, int64_t words_per_rb, const int64_t* __restrict__ rowptr,
                              const int32_t* __restrict__ col, unsigned* __restrict__ bitmap) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t I = i / R;
  unsigned* row = bitmap + I * words_per_rb;
  int64_t a = rowptr[i], b = rowptr[i + 1];
  int64_t last = -1;
  for (int64_t k = a; k < b; ++k) {
    int64_t J = col[k] / C;
    if (J != last) {
      atomicOr(row + (J >> 5), 1u << (J & 31));
      last = J;
    }
  }
}

// One warp per row block: number of tiles.
__global__ void k_tile_count(int64_t nRB, int64_t words_per_rb, const unsigned* __restrict__ bitmap,
                             int64_t* __restrict__ count) {
  int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (I >= nRB) return;
  const unsigned* row = bitmap + I * words_per_rb;
  int64_t c = 0;
  for (int64_t w = lane; w < words_per_rb; w += 32) c += __popc(row[w]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) count[I] = c;
}

// One warp per row block: write its tile column indices in ascending order.
__global__ void k_tile_fill(int64_t nRB, int64_t words_per_rb, const unsigned* __restrict__ bitmap,
                            const int64_t* __restrict__ tile_ptr, int32_t* __restrict__ tile_col) {
  int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (I >= nRB) return;
  const unsigned* row = bitmap + I * words_per_rb;
  int64_t out = tile_ptr[I];
  for (int64_t w0 = 0; w0 < words_per_rb; w0 += 32) {
    int64_t w = w0 + lane;
    unsigned bits = (w < words_per_rb) ? row[w] : 0u;
    int cnt = __popc(bits);
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int excl = incl - cnt;
    int total = __shfl_sync(0xffffffffu, incl, 31);
    int64_t pos = out + excl;
    while (bits) {
      int b = __ffs(bits) - 1;
      bits &= bits - 1;
      tile_col[pos++] = static_cast<int32_t>(w * 32 + b);
    }
    out += total;
  }
}

eig_status build_tile_lists(int64_t n, int R, int C, const int64_t* rowptr, const int32_t* col, cudaStream_t st,
                            DevBuf& tile_ptr, DevBuf& tile_col, std::vector<int64_t>& h_ptr,
                            std::vector<int32_t>& h_col) {
  const int64_t nRB = (n + R - 1) / R, nCB = (n + C - 1) / C;
  const int64_t wpr = (nCB + 31) / 32;
  const int tb = 256;
  const int64_t gb = (n + tb - 1) / tb;
  DevBuf bitmap;
  EIG_TRY(bitmap.reserve(nRB * wpr * 4));
  EIG_CUDA_TRY(cudaMemsetAsync(bitmap.p, 0, nRB * wpr * 4, st));
  k_tile_bitmap<<<(unsigned)gb, tb, 0, st>>>(n, R, C, wpr, rowptr, col, bitmap.as<unsigned>());
  EIG_LAUNCH_CHECK("k_tile_bitmap");
  DevBuf cnt;
  EIG_TRY(cnt.reserve(nRB * 8));
  const int64_t wb = (nRB * 32 + tb - 1) / tb;
  k_tile_count<<<(unsigned)wb, tb, 0, st>>>(nRB, wpr, bitmap.as<unsigned>(), cnt.as<int64_t>());
  EIG_LAUNCH_CHECK("k_tile_count");
  std::vector<int64_t> h_cnt(nRB);
  h_ptr.assign(nRB + 1, 0);
  EIG_CUDA_TRY(cudaMemcpyAsync(h_cnt.data(), cnt.p, nRB * 8, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t I = 0; I < nRB; ++I) h_ptr[I + 1] = h_ptr[I] + h_cnt[I];
  const int64_t nt = h_ptr[nRB];
  EIG_TRY(tile_ptr.reserve((nRB + 1) * 8));
  EIG_TRY(tile_col.reserve(std::max<int64_t>(nt, 1) * 4));
  EIG_CUDA_TRY(cudaMemcpyAsync(tile_ptr.p, h_ptr.data(), (nRB + 1) * 8, cudaMemcpyHostToDevice, st));
  k_tile_fill<<<(unsigned)wb, tb, 0, st>>>(nRB, wpr, bitmap.as<unsigned>(), tile_ptr.as<int64_t>(),
                                          tile_col.as<int32_t>());
  EIG_LAUNCH_CHECK("k_tile_fill");
  h_col.assign(nt, 0);
  if (nt) EIG_CUDA_TRY(cudaMemcpyAsync(h_col.data(), tile_col.p, nt * 4, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  return EIG_OK;
}

double SpmmPlan::algorithmic_bytes(int nb, size_t vb) const {
  // one read of the stored triangle (values + int32 columns) and of rowptr, X read and Y written once
  return double(nnz) * (dtype_size(val_type) + 4.0) + 8.0 * double(n + 1) + 2.0 * double(n) * nb * double(vb);
}

eig_status spmm_plan_build(SpmmPlan* P, const eig_csr_upper* H, int R, int C, int layout, int copy,
                           cudaStream_t st) {
  if (!H || H->n <= 0 || H->nnz < 0 || !H->rowptr || (!H->col && H->nnz) || (!H->val && H->nnz)) return EIG_EINVAL;
  if (H->val_type != EIG_F32 && H->val_type != EIG_F64 && H->val_type != EIG_BF16) return EIG_EINVAL;
  if (H->n > INT32_MAX) return EIG_EUNSUPPORTED;  // int32 column indices
  if (R == 0) R = 256;
  if (C == 0) C = std::min(64, R);
  if (R % 32 || C % 32 || R > 512 || C > R || R % C) return EIG_EINVAL;
  P->n = H->n; P->nnz = H->nnz; P->R = R; P->C = C; P->val_type = H->val_type;
  const int64_t n = H->n, nnz = H->nnz;
  const size_t vb = dtype_size(H->val_type);
  // matrix on the device
  if (!H->on_device || copy) {
    cudaMemcpyKind kind = H->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    EIG_TRY(P->own_rowptr.reserve((n + 1) * 8));
    EIG_TRY(P->own_col.reserve(std::max<int64_t>(nnz, 1) * 4));
    EIG_TRY(P->own_val.reserve(std::max<int64_t>(nnz, 1) * vb));
    EIG_CUDA_TRY(cudaMemcpyAsync(P->own_rowptr.p, H->rowptr, (n + 1) * 8, kind, st));
    if (nnz) {
      EIG_CUDA_TRY(cudaMemcpyAsync(P->own_col.p, H->col, nnz * 4, kind, st));
      EIG_CUDA_TRY(cudaMemcpyAsync(P->own_val.p, H->val, nnz * vb, kind, st));
    }
    P->rowptr = P->own_rowptr.as<int64_t>();
    P->col = P->own_col.as<int32_t>();
    P->val = P->own_val.p;
  } else {
    P->rowptr = H->rowptr; P->col = H->col; P->val = H->val;
  }
  // rowptr end points
  int64_t ends[2];
  EIG_CUDA_TRY(cudaMemcpyAsync(&ends[0], P->rowptr, 8, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(&ends[1], P->rowptr + n, 8, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  if (ends[0] != 0 || ends[1] != nnz) return EIG_EINVAL;
  // structure validation on the device
  DevBuf flag;
  EIG_TRY(flag.reserve(4));
  EIG_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 4, st));
  const int tb = 256;
  const int64_t gb = (n + tb - 1) / tb;
  k_validate_csr<<<(unsigned)gb, tb, 0, st>>>(n, P->rowptr, P->col, nnz, flag.as<int>());
  EIG_LAUNCH_CHECK("k_validate_csr");
  int bad = 0;
  EIG_CUDA_TRY(cudaMemcpyAsync(&bad, flag.p, 4, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  if (bad) return EIG_EINVAL;
  // diagonal (for preconditioners)
  EIG_TRY(P->diag.reserve(n * 8));
  k_extract_diag<<<(unsigned)gb, tb, 0, st>>>(n, P->rowptr, P->col, P->val, (int)H->val_type, P->diag.as<double>());
  EIG_LAUNCH_CHECK("k_extract_diag");
  // tile bitmap -> per-row-block tile lists
  P->nRB = (n + R - 1) / R;
  P->nCB = (n + C - 1) / C;
  std::vector<int64_t> h_ptr;
  std::vector<int32_t> h_col;
  EIG_TRY(build_tile_lists(n, R, C, P->rowptr, P->col, st, P->tile_ptr, P->tile_col, h_ptr, h_col));
  P->n_tiles = h_ptr[P->nRB];
  // slots for non-local tiles (column block outside the row block's own row range), and the
  // transpose schedule: a stable counting sort of the slots by column block.
  const int64_t cpr = R / C;  // column blocks per row block
  std::vector<int32_t> h_slot(P->n_tiles, -1);
  std::vector<int64_t> per_cb(P->nCB + 1, 0);
  int64_t s = 0;
  for (int64_t I = 0; I < P->nRB; ++I) {
    for (int64_t t = h_ptr[I]; t < h_ptr[I + 1]; ++t) {
      int64_t J = h_col[t];
      if (J >= (I + 1) * cpr) {
        h_slot[t] = static_cast<int32_t>(s++);
        per_cb[J + 1]++;
      }
    }
  }
  P->n_slots = s;
  if (s > INT32_MAX) return EIG_EUNSUPPORTED;
  std::vector<int32_t> h_sched_cb;
  std::vector<int64_t> h_sched_ptr(1, 0);
  for (int64_t J = 0; J < P->nCB; ++J) {
    if (per_cb[J + 1]) {
      h_sched_cb.push_back(static_cast<int32_t>(J));
      h_sched_ptr.push_back(h_sched_ptr.back() + per_cb[J + 1]);
    }
  }
  for (int64_t J = 0; J < P->nCB; ++J) per_cb[J + 1] += per_cb[J];
  std::vector<int32_t> h_sched_slot(std::max<int64_t>(s, 1));
  {
    std::vector<int64_t> fillpos(per_cb.begin(), per_cb.end() - 1);
    for (int64_t I = 0; I < P->nRB; ++I)
      for (int64_t t = h_ptr[I]; t < h_ptr[I + 1]; ++t)
        if (h_slot[t] >= 0) h_sched_slot[fillpos[h_col[t]]++] = h_slot[t];
  }
  P->n_sched = static_cast<int64_t>(h_sched_cb.size());
  EIG_TRY(P->tile_slot.reserve(std::max<int64_t>(P->n_tiles, 1) * 4));
  EIG_TRY(P->sched_ptr.reserve((P->n_sched + 1) * 8));
  EIG_TRY(P->sched_cb.reserve(std::max<int64_t>(P->n_sched, 1) * 4));
  EIG_TRY(P->sched_slot.reserve(std::max<int64_t>(s, 1) * 4));
  if (P->n_tiles)
    EIG_CUDA_TRY(cudaMemcpyAsync(P->tile_slot.p, h_slot.data(), P->n_tiles * 4, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->sched_ptr.p, h_sched_ptr.data(), (P->n_sched + 1) * 8, cudaMemcpyHostToDevice, st));
  if (P->n_sched)
    EIG_CUDA_TRY(cudaMemcpyAsync(P->sched_cb.p, h_sched_cb.data(), P->n_sched * 4, cudaMemcpyHostToDevice, st));
  if (s) EIG_CUDA_TRY(cudaMemcpyAsync(P->sched_slot.p, h_sched_slot.data(), s * 4, cudaMemcpyHostToDevice, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  P->layout = EIG_LAYOUT_CSR;
  if (layout == EIG_LAYOUT_CSR) return EIG_OK;
  bool want_mirror = (layout == EIG_LAYOUT_MIRRORED || layout == EIG_LAYOUT_AUTO) && R == 256 && C == 64;
  if (want_mirror && layout == EIG_LAYOUT_AUTO) {
    size_t fr = 0, tot = 0;
    EIG_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    want_mirror = mirror_bytes_estimate(P) < fr / 10 * 8;
  }
  if (want_mirror) {
    EIG_TRY(spmm_plan_build_mirror(P, h_ptr, h_col, st));
    P->layout = EIG_LAYOUT_MIRRORED;
    return EIG_OK;
  }
  if (C <= 256) {
    EIG_TRY(spmm_plan_build_tiled(P, 2048, st));
    P->layout = EIG_LAYOUT_HALF;
  }
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// Phase 1: per row block, gather + in-CTA transposed accumulation
// ---------------------------------------------------------------------------------------
template <typename T, typename V, int NB, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_spmm_rowblock(int64_t n, int R, int C, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                const V* __restrict__ val, const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ tile_col,
                const int32_t* __restrict__ tile_slot, const T* __restrict__ X, T* __restrict__ Y,
                T* __restrict__ Z) {
  typedef LaneShape<T, NB> S;
  constexpr int EPL = S::EPL, L = S::L, E = S::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);                 // C x NB
  T* sZ = sX + (size_t)C * NB;                            // WARPS x C x NB
  T* sY = sZ + (size_t)WARPS * C * NB;                    // R x NB
  int64_t* sCur = reinterpret_cast<int64_t*>(sY + (size_t)R * NB);  // R
  int64_t* sEnd = sCur + R;                               // R

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t I = blockIdx.x;
  const int64_t r0 = I * R;
  const int rows = (int)min64(R, n - r0);
  const int RPW = R / WARPS;
  const int q = lane % L;          // 16-byte slice of the row this lane handles
  const int eg = lane / L;         // entry group within a warp step

  for (int i = tid; i < WARPS * C * NB; i += WARPS * 32) sZ[i] = T(0);
  for (int i = tid; i < R * NB; i += WARPS * 32) sY[i] = T(0);
  for (int i = tid; i < R; i += WARPS * 32) {
    if (i < rows) { sCur[i] = rowptr[r0 + i]; sEnd[i] = rowptr[r0 + i + 1]; }
    else { sCur[i] = 0; sEnd[i] = 0; }
  }

  const int64_t t0 = tile_ptr[I], t1 = tile_ptr[I + 1];
  T* sZw = sZ + (size_t)w * C * NB;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t J = tile_col[t];
    const int64_t cb0 = J * C;
    const bool local = (cb0 < r0 + R);
    // stage X_J (zero beyond n)
    {
      const int64_t avail = min64(C, n - cb0);
      for (int i = tid; i < C * NB / EPL; i += WARPS * 32) {
        const int rr = (i * EPL) / NB;
        Vec<T, EPL> v;
        if (rr < avail) v = VecIO<T, EPL>::ld(X + (cb0 + rr) * NB + (i * EPL) % NB);
        else v.zero();
        VecIO<T, EPL>::st(sX + (size_t)i * EPL, v);
      }
    }
    __syncthreads();
    const int64_t climit = cb0 + C;
    for (int rl = w * RPW; rl < (w + 1) * RPW && rl < rows; ++rl) {
      int64_t cur = sCur[rl];
      const int64_t end = sEnd[rl];
      if (cur >= end) continue;
      if ((int64_t)col[cur] >= climit) continue;
      const int64_t r = r0 + rl;
      const Vec<T, EPL> xr = VecIO<T, EPL>::ld(X + r * NB + q * EPL);
      Vec<T, EPL> yacc;
      yacc.zero();
      while (cur < end) {
        const int64_t idx = cur + lane;
        const bool valid = idx < end;
        int c = valid ? col[idx] : INT32_MAX;
        T v = valid ? (T)ValLoad<V>::get(val, idx) : T(0);
        const bool in = valid && (c < climit);
        const unsigned m = __ballot_sync(0xffffffffu, in);
        const int cnt = __popc(m);
        for (int s0 = 0; s0 < cnt; s0 += E) {
          const int e = s0 + eg;
          const int ce = __shfl_sync(0xffffffffu, c, e & 31);
          const T ve = __shfl_sync(0xffffffffu, v, e & 31);
          if (e < cnt) {
            const int lc = ce - (int)cb0;
            const Vec<T, EPL> xc = VecIO<T, EPL>::ld(sX + (size_t)lc * NB + q * EPL);
#pragma unroll
            for (int k = 0; k < EPL; ++k) yacc.v[k] = fma(ve, xc.v[k], yacc.v[k]);
            if (!(local && (int64_t)ce == r)) {
              T* zp = sZw + (size_t)lc * NB + q * EPL;
              Vec<T, EPL> z = VecIO<T, EPL>::ld(zp);
#pragma unroll
              for (int k = 0; k < EPL; ++k) z.v[k] = fma(ve, xr.v[k], z.v[k]);
              VecIO<T, EPL>::st(zp, z);
            }
          }
        }
        cur += cnt;
        if (cnt < 32) break;
      }
#pragma unroll
      for (int o = L; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < EPL; ++k) yacc.v[k] += __shfl_xor_sync(0xffffffffu, yacc.v[k], o);
      }
      if (lane < L) {
        T* yp = sY + (size_t)rl * NB + lane * EPL;
        Vec<T, EPL> y = VecIO<T, EPL>::ld(yp);
#pragma unroll
        for (int k = 0; k < EPL; ++k) y.v[k] += yacc.v[k];
        VecIO<T, EPL>::st(yp, y);
      }
      if (lane == 0) sCur[rl] = cur;
    }
    __syncthreads();
    // fixed-order sum of the warps' private transposed partials
    const int32_t slot = tile_slot[t];
    const int64_t yoff = cb0 - r0;   // local: row offset of this column block in the CTA's y
    for (int i = tid; i < C * NB; i += WARPS * 32) {
      T acc = T(0);
#pragma unroll
      for (int ww = 0; ww < WARPS; ++ww) {
        acc += sZ[(size_t)ww * C * NB + i];
        sZ[(size_t)ww * C * NB + i] = T(0);
      }
      if (local) {
        const int64_t rr = yoff + i / NB;
        if (rr < rows) sY[rr * NB + i % NB] += acc;
      } else {
        Z[(size_t)slot * C * NB + i] = acc;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < rows * NB / EPL; i += WARPS * 32) {
    Vec<T, EPL> v = VecIO<T, EPL>::ld(sY + (size_t)i * EPL);
    VecIO<T, EPL>::st(Y + r0 * NB + (size_t)i * EPL, v);
  }
}

// ---------------------------------------------------------------------------------------
// Phase 2: Y_J += sum of the scratch slots of column block J, in schedule order
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
__global__ void k_spmm_transpose_reduce(int64_t n, int C, const int64_t* __restrict__ sched_ptr,
                                        const int32_t* __restrict__ sched_cb, const int32_t* __restrict__ sched_slot,
                                        const T* __restrict__ Z, T* __restrict__ Y) {
  constexpr int EPL = LaneShape<T, NB>::EPL;
  const int64_t b = blockIdx.x;
  const int64_t J = sched_cb[b];
  const int64_t s0 = sched_ptr[b], s1 = sched_ptr[b + 1];
  const int64_t cb0 = J * C;
  const int64_t avail = min64(C, n - cb0);
  for (int i = threadIdx.x; i < C * NB / EPL; i += blockDim.x) {
    const int64_t rr = (int64_t)(i * EPL) / NB;
    if (rr >= avail) continue;
    T* yp = Y + cb0 * NB + (size_t)i * EPL;
    Vec<T, EPL> acc = VecIO<T, EPL>::ld(yp);
    for (int64_t s = s0; s < s1; ++s) {
      const Vec<T, EPL> z = VecIO<T, EPL>::ld(Z + (size_t)sched_slot[s] * C * NB + (size_t)i * EPL);
#pragma unroll
      for (int k = 0; k < EPL; ++k) acc.v[k] += z.v[k];
    }
    VecIO<T, EPL>::st(yp, acc);
  }
}

// ---------------------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------------------
template <typename T, int NB>
static size_t smem_bytes(const SpmmPlan* P, int warps) {
  return ((size_t)P->C * NB + (size_t)warps * P->C * NB + (size_t)P->R * NB) * sizeof(T) + 2 * 8 * (size_t)P->R;
}

size_t spmm_scratch_bytes(const SpmmPlan* P, int nb, eig_dtype vt) {
  if (P->mirrored) return 16;
  return (size_t)std::max<int64_t>(P->n_slots, 1) * P->C * nb * dtype_size(vt);
}

template <typename T, typename V, int NB, int WARPS>
static eig_status launch_rowblock(SpmmPlan* P, const T* X, T* Y, T* Z, size_t sm, cudaStream_t st) {
  auto kern = k_spmm_rowblock<T, V, NB, WARPS>;
  EIG_CUDA_TRY(::eig::ensure_dyn_smem(kern, (int)sm));
  kern<<<(unsigned)P->nRB, WARPS * 32, sm, st>>>(P->n, P->R, P->C, P->rowptr, P->col,
                                                 static_cast<const V*>(P->val), P->tile_ptr.as<int64_t>(),
                                                 P->tile_col.as<int32_t>(), P->tile_slot.as<int32_t>(), X, Y, Z);
  EIG_LAUNCH_CHECK("k_spmm_rowblock");
  return EIG_OK;
}

template <typename T, int NB>
eig_status transpose_reduce_launch(SpmmPlan* P, const T* Z, T* Y, cudaStream_t st) {
  if (P->n_sched) {
    k_spmm_transpose_reduce<T, NB><<<(unsigned)P->n_sched, 256, 0, st>>>(
        P->n, P->C, P->sched_ptr.as<int64_t>(), P->sched_cb.as<int32_t>(), P->sched_slot.as<int32_t>(), Z, Y);
    EIG_LAUNCH_CHECK("k_spmm_transpose_reduce");
  }
  return EIG_OK;
}
#define EIG_TR_INST(T)                                                                   \
  template eig_status transpose_reduce_launch<T, 1>(SpmmPlan*, const T*, T*, cudaStream_t);  \
  template eig_status transpose_reduce_launch<T, 2>(SpmmPlan*, const T*, T*, cudaStream_t);  \
  template eig_status transpose_reduce_launch<T, 4>(SpmmPlan*, const T*, T*, cudaStream_t);  \
  template eig_status transpose_reduce_launch<T, 8>(SpmmPlan*, const T*, T*, cudaStream_t);  \
  template eig_status transpose_reduce_launch<T, 16>(SpmmPlan*, const T*, T*, cudaStream_t); \
  template eig_status transpose_reduce_launch<T, 32>(SpmmPlan*, const T*, T*, cudaStream_t);
EIG_TR_INST(float)
EIG_TR_INST(double)

template <typename T, typename V, int NB> eig_status tiled_launch(SpmmPlan* P, const T* X, T* Y, T* Z, cudaStream_t st);
template <typename T, typename V, int NB> eig_status mirror_launch(SpmmPlan* P, const T* X, T* Y, cudaStream_t st);

template <typename T, typename V, int NB>
eig_status mirror_launch_cheb(SpmmPlan* P, const T* X, T* Y, const T* Qp, const int* active, double alpha, double c,
                              int first, cudaStream_t st);

template <typename T, typename V, int NB>
static eig_status launch(SpmmPlan* P, const T* X, T* Y, T* Z, cudaStream_t st) {
  // gather-only kernel on the mirrored copy (its stages fit in shared memory for every
  // supported shape; it needs no scratch)
  if (P->mirrored) return mirror_launch<T, V, NB>(P, X, Y, st);
  if (P->tiled) {
    // the tile-contiguous kernel; when its stages do not fit in shared memory (wide FP64
    // blocks) the CSR kernel below computes the same product
    const eig_status s = tiled_launch<T, V, NB>(P, X, Y, Z, st);
    if (s != EIG_EUNSUPPORTED) return s;
  }
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem_bytes<T, NB>(P, 4) <= (size_t)maxsm) {
    EIG_TRY((launch_rowblock<T, V, NB, 4>(P, X, Y, Z, smem_bytes<T, NB>(P, 4), st)));
  } else if (smem_bytes<T, NB>(P, 2) <= (size_t)maxsm) {
    EIG_TRY((launch_rowblock<T, V, NB, 2>(P, X, Y, Z, smem_bytes<T, NB>(P, 2), st)));
  } else {
    return EIG_EUNSUPPORTED;
  }
  return transpose_reduce_launch<T, NB>(P, Z, Y, st);
}

template <typename T, typename V, int NB, bool CHEB>
eig_status mirror_launch_batch(const SpmmJob* jobs, int count, cudaStream_t st);

eig_status spmm_run_batch(const SpmmJob* jobs, int count, int nb, eig_dtype vt, bool cheb, cudaStream_t st) {
  if (count < 1 || !jobs) return EIG_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!jobs[i].P || !jobs[i].P->mirrored || jobs[i].P->val_type != EIG_F32) return EIG_EUNSUPPORTED;
  if (nb != 8 && nb != 16) return EIG_EUNSUPPORTED;
  if (vt == EIG_F32) {
    if (nb == 8) return cheb ? mirror_launch_batch<float, float, 8, true>(jobs, count, st)
                             : mirror_launch_batch<float, float, 8, false>(jobs, count, st);
    return cheb ? mirror_launch_batch<float, float, 16, true>(jobs, count, st)
                : mirror_launch_batch<float, float, 16, false>(jobs, count, st);
  }
  if (vt == EIG_F64) {
    if (nb == 8) return cheb ? mirror_launch_batch<double, float, 8, true>(jobs, count, st)
                             : mirror_launch_batch<double, float, 8, false>(jobs, count, st);
    return cheb ? mirror_launch_batch<double, float, 16, true>(jobs, count, st)
                : mirror_launch_batch<double, float, 16, false>(jobs, count, st);
  }
  return EIG_EUNSUPPORTED;
}

template <typename T, typename V>
eig_status mirror_launch_column(SpmmPlan* P, const T* X, T* Y, int ld, int col, cudaStream_t st);

template <typename T, typename V>
static eig_status dispatch_nb(SpmmPlan* P, const T* X, T* Y, T* Z, int nb, cudaStream_t st) {
  switch (nb) {
    case 1: return launch<T, V, 1>(P, X, Y, Z, st);
    case 2: return launch<T, V, 2>(P, X, Y, Z, st);
    case 4: return launch<T, V, 4>(P, X, Y, Z, st);
    case 8: return launch<T, V, 8>(P, X, Y, Z, st);
    case 16: return launch<T, V, 16>(P, X, Y, Z, st);
    case 32: return launch<T, V, 32>(P, X, Y, Z, st);
    default: return EIG_EINVAL;
  }
}

eig_status spmm_run_with_scratch(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, void* scratch,
                                 cudaStream_t st) {
  if (!P || !X || !Y) return EIG_EINVAL;
  if (vt != EIG_F32 && vt != EIG_F64) return EIG_EINVAL;
  // every kernel moves X and Y rows in pieces of min(16, nb * element size) bytes
  const uintptr_t align = (uintptr_t)std::min<size_t>(16, (size_t)nb * dtype_size(vt));
  if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & (align - 1)) return EIG_EINVAL;
  if (vt == EIG_F32) {
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    float* z = static_cast<float*>(scratch);
    if (P->val_type == EIG_F32) return dispatch_nb<float, float>(P, x, y, z, nb, st);
    if (P->val_type == EIG_BF16) return dispatch_nb<float, uint16_t>(P, x, y, z, nb, st);
    return EIG_EUNSUPPORTED;
  }
  if (vt == EIG_F64) {
    const double* x = static_cast<const double*>(X);
    double* y = static_cast<double*>(Y);
    double* z = static_cast<double*>(scratch);
    if (P->val_type == EIG_F64) return dispatch_nb<double, double>(P, x, y, z, nb, st);
    if (P->val_type == EIG_F32) return dispatch_nb<double, float>(P, x, y, z, nb, st);
    if (P->val_type == EIG_BF16) return dispatch_nb<double, uint16_t>(P, x, y, z, nb, st);
    return EIG_EUNSUPPORTED;
  }
  return EIG_EINVAL;
}

eig_status spmm_run_column(SpmmPlan* P, const void* X, void* Y, int ld, int col, eig_dtype vt, cudaStream_t st) {
  if (!P || !X || !Y || ld < 1 || col < 0 || col >= ld) return EIG_EINVAL;
  if (!P->mirrored) return EIG_EUNSUPPORTED;
  if (vt == EIG_F32) {
    const float* x = static_cast<const float*>(X);
    float* y = static_cast<float*>(Y);
    if (P->val_type == EIG_F32) return mirror_launch_column<float, float>(P, x, y, ld, col, st);
    if (P->val_type == EIG_BF16) return mirror_launch_column<float, uint16_t>(P, x, y, ld, col, st);
    return EIG_EUNSUPPORTED;
  }
  if (vt == EIG_F64) {
    const double* x = static_cast<const double*>(X);
    double* y = static_cast<double*>(Y);
    if (P->val_type == EIG_F64) return mirror_launch_column<double, double>(P, x, y, ld, col, st);
    if (P->val_type == EIG_F32) return mirror_launch_column<double, float>(P, x, y, ld, col, st);
    if (P->val_type == EIG_BF16) return mirror_launch_column<double, uint16_t>(P, x, y, ld, col, st);
    return EIG_EUNSUPPORTED;
  }
  return EIG_EINVAL;
}

eig_status spmm_run(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, cudaStream_t st) {
  if (!P) return EIG_EINVAL;
  if (nb != 1 && nb != 2 && nb != 4 && nb != 8 && nb != 16 && nb != 32) return EIG_EINVAL;
  EIG_TRY(P->scratch.reserve(spmm_scratch_bytes(P, nb, vt)));
  return spmm_run_with_scratch(P, X, Y, nb, vt, P->scratch.p, st);
}

}  // namespace eig

namespace eig {

eig_status spmm_run_cheb(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, const void* Qp, const int* active,
                         double alpha, double c, int first, cudaStream_t st) {
  if (!P || !X || !Y || !active || (!first && !Qp)) return EIG_EINVAL;
  if (!P->mirrored || (nb != 8 && nb != 16 && nb != 32)) return EIG_EUNSUPPORTED;
  const size_t es = vt == EIG_F64 ? 8 : 4;
  const size_t al = std::min<size_t>(16, (size_t)nb * es);
  const uintptr_t m = (uintptr_t)X | (uintptr_t)Y | (first ? 0 : (uintptr_t)Qp);
  if (m % al) return EIG_EINVAL;
#define EIG_CHEB_NB(T, V)                                                                                            \
  switch (nb) {                                                                                                     \
    case 8: return mirror_launch_cheb<T, V, 8>(P, (const T*)X, (T*)Y, (const T*)Qp, active, alpha, c, first, st);  \
    case 16: return mirror_launch_cheb<T, V, 16>(P, (const T*)X, (T*)Y, (const T*)Qp, active, alpha, c, first, st); \
    default: return mirror_launch_cheb<T, V, 32>(P, (const T*)X, (T*)Y, (const T*)Qp, active, alpha, c, first, st); \
  }
  if (vt == EIG_F32 && P->val_type == EIG_F32) { EIG_CHEB_NB(float, float) }
  if (vt == EIG_F64 && P->val_type == EIG_F64) { EIG_CHEB_NB(double, double) }
  if (vt == EIG_F64 && P->val_type == EIG_F32) { EIG_CHEB_NB(double, float) }
#undef EIG_CHEB_NB
  return EIG_EUNSUPPORTED;
}

}  // namespace eig
