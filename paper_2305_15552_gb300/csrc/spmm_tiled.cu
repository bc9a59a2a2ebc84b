// Tile-contiguous half-stored SpMM: Y = H X, H = U + U_strict^T (Sec. 1; Eqs. upd1-upd2; half
// storage of Sec. 3.1), GB300 layout.
//
// At plan time the stored triangle is copied into chunks: a chunk holds whole rows of one tile
// (row block I x column block J), its entries contiguous as (uint8 column inside the tile,
// value) and its row offsets as uint16, every array 16-byte aligned.  A CTA owns a row block
// and streams its chunks through shared memory with 1-D bulk copies (TMA, cp.async.bulk) on a
// two-stage mbarrier pipeline: while the warps work on chunk k, the copy engine fetches chunk
// k+1 (entries, row offsets and the X_J tile it multiplies).  The arithmetic is that of the
// CSR kernel (spmm.cu): gather y_r += v X_J[c] per row, warp-private transposed partials
// z_c += v X_I[r], a fixed-order sum of the partials per tile into the CTA's y (tiles inside
// the row block) or into a scratch slot, and the transpose-schedule reduction of the slots.
// Compared with the CSR copy the stored triangle takes 5 bytes per nonzero (FP32) instead of
// 8, and no global-memory latency sits in the inner loop.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "spmm.cuh"
#include "tma.cuh"
#include "vec.cuh"

namespace eig {

// ---------------------------------------------------------------------------------------
// plan construction
// ---------------------------------------------------------------------------------------
// Thread per row: entries of row r in tile t (tiles of its row block in ascending J).
__global__ void k_tile_row_counts(int64_t n, int R, int C, const int64_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const int64_t* __restrict__ tile_ptr,
                                  const int32_t* __restrict__ tile_col, int32_t* __restrict__ cnt) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t I = r / R;
  const int rl = (int)(r - I * R);
  int64_t t = tile_ptr[I];
  const int64_t tend = tile_ptr[I + 1];
  int run = 0;
  int64_t tcur = -1;
  for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    const int J = col[k] / C;
    while (t < tend && tile_col[t] < J) ++t;
    if (t != tcur) {
      if (tcur >= 0) cnt[tcur * R + rl] = run;
      tcur = t;
      run = 0;
    }
    ++run;
  }
  if (tcur >= 0) cnt[tcur * R + rl] = run;
}

template <typename V>
__global__ void k_tile_scatter(int64_t n, int R, int C, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const V* __restrict__ val,
                               const int64_t* __restrict__ tile_ptr, const int32_t* __restrict__ tile_col,
                               const int64_t* __restrict__ dst, uint8_t* __restrict__ tcol, V* __restrict__ tval) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t I = r / R;
  const int rl = (int)(r - I * R);
  int64_t t = tile_ptr[I];
  const int64_t tend = tile_ptr[I + 1];
  int64_t pos = -1, tcur = -1;
  for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
    const int c = col[k];
    const int J = c / C;
    while (t < tend && tile_col[t] < J) ++t;
    if (t != tcur) {
      tcur = t;
      pos = dst[t * R + rl];
    }
    tcol[pos] = (uint8_t)(c - J * C);
    tval[pos] = val[k];
    ++pos;
  }
}

eig_status spmm_plan_build_tiled(SpmmPlan* P, int cap, cudaStream_t st) {
  const int R = P->R, C = P->C;
  if (C > 256 || R > 4096) return EIG_EUNSUPPORTED;
  cap = std::max(cap, 256);
  cap = (cap + 15) / 16 * 16;
  P->cap = cap;
  const int64_t n = P->n, nt = P->n_tiles;
  const int tb = 256;
  const int64_t gb = (n + tb - 1) / tb;
  DevBuf dcnt;
  EIG_TRY(dcnt.reserve(std::max<int64_t>(nt, 1) * R * 4));
  EIG_CUDA_TRY(cudaMemsetAsync(dcnt.p, 0, std::max<int64_t>(nt, 1) * R * 4, st));
  k_tile_row_counts<<<(unsigned)gb, tb, 0, st>>>(n, R, C, P->rowptr, P->col, P->tile_ptr.as<int64_t>(),
                                                 P->tile_col.as<int32_t>(), dcnt.as<int32_t>());
  EIG_LAUNCH_CHECK("k_tile_row_counts");
  std::vector<int32_t> cnt((size_t)nt * R);
  std::vector<int64_t> tptr(P->nRB + 1);
  std::vector<int32_t> tcolh(nt), tslot(nt);
  if (nt) {
    EIG_CUDA_TRY(cudaMemcpyAsync(cnt.data(), dcnt.p, (size_t)nt * R * 4, cudaMemcpyDeviceToHost, st));
    EIG_CUDA_TRY(cudaMemcpyAsync(tcolh.data(), P->tile_col.p, nt * 4, cudaMemcpyDeviceToHost, st));
    EIG_CUDA_TRY(cudaMemcpyAsync(tslot.data(), P->tile_slot.p, nt * 4, cudaMemcpyDeviceToHost, st));
  }
  EIG_CUDA_TRY(cudaMemcpyAsync(tptr.data(), P->tile_ptr.p, (P->nRB + 1) * 8, cudaMemcpyDeviceToHost, st));
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  dcnt.release();
  // greedy chunking of every tile's rows (trimmed to its first..last nonempty row)
  std::vector<TileChunk> ch;
  std::vector<int64_t> cptr(P->nRB + 1, 0);
  std::vector<uint16_t> rp;
  std::vector<int64_t> dst((size_t)nt * R, -1);
  int64_t ent = 0;
  for (int64_t I = 0; I < P->nRB; ++I) {
    const int rows = (int)std::min<int64_t>(R, n - I * R);
    for (int64_t t = tptr[I]; t < tptr[I + 1]; ++t) {
      const int32_t* c = cnt.data() + (size_t)t * R;
      int first = 0, last = rows - 1;
      while (first < rows && c[first] == 0) ++first;
      while (last >= first && c[last] == 0) --last;
      if (first > last) continue;
      int ra = first;
      bool first_chunk = true;
      while (ra <= last) {
        int rb = ra;
        int64_t tot = 0;
        while (rb <= last && (tot + c[rb] <= cap || rb == ra)) tot += c[rb++];
        TileChunk k;
        k.ent_off = ent;
        k.nent_pad = (int32_t)((tot + 15) / 16 * 16);
        k.J = tcolh[t];
        k.rp_off = (int32_t)rp.size();
        k.ra = (int16_t)ra;
        k.rb = (int16_t)rb;
        k.slot = tslot[t];
        k.flags = (first_chunk ? 1 : 0) | (rb > last ? 2 : 0);
        int64_t off = 0;
        for (int r = ra; r < rb; ++r) {
          rp.push_back((uint16_t)off);
          dst[(size_t)t * R + r] = ent + off;
          off += c[r];
        }
        rp.push_back((uint16_t)off);
        while (rp.size() % 8) rp.push_back((uint16_t)off);
        ent += k.nent_pad;
        ch.push_back(k);
        first_chunk = false;
        ra = rb;
      }
    }
    cptr[I + 1] = (int64_t)ch.size();
  }
  if (rp.size() > (size_t)INT32_MAX) return EIG_EUNSUPPORTED;
  P->n_chunks = (int64_t)ch.size();
  P->tiled_entries = ent;
  P->tiled_rp = (int64_t)rp.size();
  const size_t vb = dtype_size(P->val_type);
  EIG_TRY(P->chunk_ptr.reserve((P->nRB + 1) * 8));
  EIG_TRY(P->chunks.reserve(std::max<size_t>(ch.size(), 1) * sizeof(TileChunk)));
  EIG_TRY(P->trp.reserve(std::max<size_t>(rp.size(), 8) * 2));
  EIG_TRY(P->tcol.reserve(std::max<int64_t>(ent, 16)));
  EIG_TRY(P->tval.reserve(std::max<int64_t>(ent, 16) * vb));
  EIG_TRY(P->err.reserve(16));
  EIG_CUDA_TRY(cudaMemsetAsync(P->err.p, 0, 16, st));
  EIG_CUDA_TRY(cudaMemsetAsync(P->tcol.p, 0, std::max<int64_t>(ent, 16), st));
  EIG_CUDA_TRY(cudaMemsetAsync(P->tval.p, 0, std::max<int64_t>(ent, 16) * vb, st));
  EIG_CUDA_TRY(cudaMemcpyAsync(P->chunk_ptr.p, cptr.data(), (P->nRB + 1) * 8, cudaMemcpyHostToDevice, st));
  if (!ch.empty())
    EIG_CUDA_TRY(cudaMemcpyAsync(P->chunks.p, ch.data(), ch.size() * sizeof(TileChunk), cudaMemcpyHostToDevice, st));
  if (!rp.empty()) EIG_CUDA_TRY(cudaMemcpyAsync(P->trp.p, rp.data(), rp.size() * 2, cudaMemcpyHostToDevice, st));
  DevBuf ddst;
  EIG_TRY(ddst.reserve(std::max<size_t>(dst.size(), 1) * 8));
  if (!dst.empty()) EIG_CUDA_TRY(cudaMemcpyAsync(ddst.p, dst.data(), dst.size() * 8, cudaMemcpyHostToDevice, st));
  if (P->val_type == EIG_F32)
    k_tile_scatter<float><<<(unsigned)gb, tb, 0, st>>>(n, R, C, P->rowptr, P->col, (const float*)P->val,
                                                       P->tile_ptr.as<int64_t>(), P->tile_col.as<int32_t>(),
                                                       ddst.as<int64_t>(), P->tcol.as<uint8_t>(), P->tval.as<float>());
  else if (P->val_type == EIG_F64)
    k_tile_scatter<double><<<(unsigned)gb, tb, 0, st>>>(n, R, C, P->rowptr, P->col, (const double*)P->val,
                                                        P->tile_ptr.as<int64_t>(), P->tile_col.as<int32_t>(),
                                                        ddst.as<int64_t>(), P->tcol.as<uint8_t>(),
                                                        P->tval.as<double>());
  else
    k_tile_scatter<uint16_t><<<(unsigned)gb, tb, 0, st>>>(n, R, C, P->rowptr, P->col, (const uint16_t*)P->val,
                                                          P->tile_ptr.as<int64_t>(), P->tile_col.as<int32_t>(),
                                                          ddst.as<int64_t>(), P->tcol.as<uint8_t>(),
                                                          P->tval.as<uint16_t>());
  EIG_LAUNCH_CHECK("k_tile_scatter");
  EIG_CUDA_TRY(cudaStreamSynchronize(st));
  P->tiled = true;
  return EIG_OK;
}

// ---------------------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------------------
struct TiledArgs {
  int64_t n;
  int R, C, cap, rp_cap;
  const int64_t* chunk_ptr;
  const TileChunk* chunks;
  const uint8_t* tcol;
  const void* tval;
  const uint16_t* trp;
  int* err;
};

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~size_t(127); }

template <typename T, typename V>
struct StageLayout {
  size_t col, val, rp, xj, bytes;
  __host__ __device__ StageLayout(int cap, int rp_cap, int C, int NB) {
    col = 0;
    val = align128((size_t)cap);
    rp = val + align128((size_t)cap * sizeof(V));
    xj = rp + align128((size_t)rp_cap * 2);
    bytes = xj + align128((size_t)C * NB * sizeof(T));
  }
};

template <typename T, typename V, int NB, int WARPS>
__global__ void __launch_bounds__(WARPS * 32)
k_spmm_tiled(TiledArgs a, const T* __restrict__ X, T* __restrict__ Y, T* __restrict__ Z) {
  typedef LaneShape<T, NB> S;
  constexpr int EPL = S::EPL, L = S::L, E = S::E;
  typedef typename ValLoad<V>::storage VS;
  constexpr bool kXjBulk = (NB * sizeof(T)) % 16 == 0;
  extern __shared__ __align__(128) unsigned char smem[];
  const StageLayout<T, V> SL(a.cap, a.rp_cap, a.C, NB);
  unsigned char* stage[2] = {smem, smem + SL.bytes};
  T* sZ = reinterpret_cast<T*>(smem + 2 * SL.bytes);              // WARPS x C x NB
  T* sY = sZ + (size_t)WARPS * a.C * NB;                          // R x NB
  T* sXI = sY + (size_t)a.R * NB;                                 // R x NB: this row block's X rows
  uint64_t* bar = reinterpret_cast<uint64_t*>(sXI + (size_t)a.R * NB);
  __shared__ int s_abort;

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t I = blockIdx.x;
  const int64_t r0 = I * a.R;
  const int rows = (int)min64(a.R, a.n - r0);
  const int q = lane % L, eg = lane / L;
  const int64_t c0 = a.chunk_ptr[I], c1 = a.chunk_ptr[I + 1];
  const V* tval = static_cast<const V*>(a.tval);

  for (int i = tid; i < WARPS * a.C * NB; i += WARPS * 32) sZ[i] = T(0);
  for (int i = tid; i < a.R * NB; i += WARPS * 32) sY[i] = T(0);
  if (tid == 0) {
    s_abort = 0;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    mbar_init_fence();
  }
  __syncthreads();
  // X_I (the row block's own rows, the operand of the transposed half) once per CTA
  if (kXjBulk) {
    if (tid == 0) {
      const uint32_t b = (uint32_t)((size_t)rows * NB * sizeof(T));
      mbar_arrive_expect_tx(&bar[2], b);
      tma_load_1d(sXI, X + r0 * NB, b, &bar[2]);
    }
  } else {
    for (int i = tid; i < rows * NB; i += WARPS * 32) sXI[i] = X[r0 * NB + i];
  }

  // bulk copies of chunk k into stage s (thread 0)
  auto issue = [&](int64_t k, int s) {
    const TileChunk ck = a.chunks[k];
    const int nr = ck.rb - ck.ra;
    const uint32_t rp_bytes = (uint32_t)(((nr + 1 + 7) / 8) * 8 * 2);
    const int64_t cb0 = (int64_t)ck.J * a.C;
    const int64_t avail = min64(a.C, a.n - cb0);
    uint32_t xj_bytes = 0;
    if (kXjBulk) xj_bytes = (uint32_t)(avail * NB * sizeof(T));
    const uint32_t bytes = (uint32_t)ck.nent_pad * (1u + (uint32_t)sizeof(VS)) + rp_bytes + xj_bytes;
    mbar_arrive_expect_tx(&bar[s], bytes);
    unsigned char* st = stage[s];
    tma_load_1d(st + SL.col, a.tcol + ck.ent_off, (uint32_t)ck.nent_pad, &bar[s]);
    tma_load_1d(st + SL.val, tval + ck.ent_off, (uint32_t)ck.nent_pad * (uint32_t)sizeof(VS), &bar[s]);
    tma_load_1d(st + SL.rp, a.trp + ck.rp_off, rp_bytes, &bar[s]);
    if (kXjBulk) tma_load_1d(st + SL.xj, X + cb0 * NB, xj_bytes, &bar[s]);
  };
  int issued[2] = {0, 0}, consumed[2] = {0, 0};  // meaningful in thread 0 only
  if (tid == 0) {
    if (c0 < c1) { issue(c0, 0); issued[0]++; }
    if (c0 + 1 < c1) { issue(c0 + 1, 1); issued[1]++; }
  }
  if (kXjBulk && !mbar_wait_bounded(&bar[2], 0)) {
    atomicOr(a.err, 2);
    s_abort = 1;
  }
  __syncthreads();
  T* sZw = sZ + (size_t)w * a.C * NB;
  for (int64_t k = c0; k < c1 && !s_abort; ++k) {
    const int s = (int)((k - c0) & 1);
    const uint32_t phase = (uint32_t)(((k - c0) >> 1) & 1);
    const TileChunk ck = a.chunks[k];
    const int64_t cb0 = (int64_t)ck.J * a.C;
    const int64_t avail = min64(a.C, a.n - cb0);
    unsigned char* st = stage[s];
    const uint8_t* scol = st + SL.col;
    const VS* sval = reinterpret_cast<const VS*>(st + SL.val);
    const uint16_t* srp = reinterpret_cast<const uint16_t*>(st + SL.rp);
    T* sX = reinterpret_cast<T*>(st + SL.xj);
    if (!kXjBulk) {
      for (int i = tid; i < a.C * NB; i += WARPS * 32) sX[i] = (i / NB < avail) ? X[cb0 * NB + i] : T(0);
    } else if (avail < a.C) {
      for (int i = (int)avail * NB + tid; i < a.C * NB; i += WARPS * 32) sX[i] = T(0);
    }
    if (!mbar_wait_bounded(&bar[s], phase)) {
      atomicOr(a.err, 1);
      s_abort = 1;
    }
    if (tid == 0) consumed[s]++;
    __syncthreads();
    if (s_abort) break;
    const bool local = cb0 < r0 + a.R;
    const int nr = ck.rb - ck.ra;
    for (int i = w; i < nr; i += WARPS) {
      const int rl = ck.ra + i;
      const int64_t r = r0 + rl;
      const int beg = srp[i], end = srp[i + 1];
      if (beg == end) continue;
      const Vec<T, EPL> xr = VecIO<T, EPL>::ld(sXI + (size_t)rl * NB + q * EPL);
      Vec<T, EPL> yacc;
      yacc.zero();
      for (int e0 = beg; e0 < end; e0 += E) {
        const int e = e0 + eg;
        if (e < end) {
          const int lc = scol[e];
          const T ve = (T)ValSmem<V>::get(sval, e);
          const Vec<T, EPL> xc = VecIO<T, EPL>::ld(sX + (size_t)lc * NB + q * EPL);
#pragma unroll
          for (int kk = 0; kk < EPL; ++kk) yacc.v[kk] = fma(ve, xc.v[kk], yacc.v[kk]);
          if (!(local && cb0 + lc == r)) {
            T* zp = sZw + (size_t)lc * NB + q * EPL;
            Vec<T, EPL> z = VecIO<T, EPL>::ld(zp);
#pragma unroll
            for (int kk = 0; kk < EPL; ++kk) z.v[kk] = fma(ve, xr.v[kk], z.v[kk]);
            VecIO<T, EPL>::st(zp, z);
          }
        }
      }
#pragma unroll
      for (int o = L; o < 32; o <<= 1) {
#pragma unroll
        for (int kk = 0; kk < EPL; ++kk) yacc.v[kk] += __shfl_xor_sync(0xffffffffu, yacc.v[kk], o);
      }
      if (lane < L) {
        T* yp = sY + (size_t)rl * NB + lane * EPL;
        Vec<T, EPL> y = VecIO<T, EPL>::ld(yp);
#pragma unroll
        for (int kk = 0; kk < EPL; ++kk) y.v[kk] += yacc.v[kk];
        VecIO<T, EPL>::st(yp, y);
      }
    }
    __syncthreads();
    if (ck.flags & 2) {
      // fixed-order sum of the warps' transposed partials of this tile
      const int64_t yoff = cb0 - r0;
      for (int i = tid; i < a.C * NB; i += WARPS * 32) {
        T acc = T(0);
#pragma unroll
        for (int ww = 0; ww < WARPS; ++ww) {
          acc += sZ[(size_t)ww * a.C * NB + i];
          sZ[(size_t)ww * a.C * NB + i] = T(0);
        }
        if (local) {
          const int64_t rr = yoff + i / NB;
          if (rr < rows) sY[rr * NB + i % NB] += acc;
        } else {
          Z[(size_t)ck.slot * a.C * NB + i] = acc;
        }
      }
      __syncthreads();
    }
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
  for (int i = tid; i < rows * NB / EPL; i += WARPS * 32) {
    Vec<T, EPL> v = VecIO<T, EPL>::ld(sY + (size_t)i * EPL);
    VecIO<T, EPL>::st(Y + r0 * NB + (size_t)i * EPL, v);
  }
}

template <typename T, typename V, int NB, int WARPS>
static size_t tiled_smem(const SpmmPlan* P) {
  const int rp_cap = (P->R + 1 + 7) / 8 * 8;
  const StageLayout<T, V> SL(P->cap, rp_cap, P->C, NB);
  return 2 * SL.bytes + ((size_t)WARPS * P->C * NB + 2 * (size_t)P->R * NB) * sizeof(T) + 4 * 8;
}

template <typename T, int NB> eig_status transpose_reduce_launch(SpmmPlan* P, const T* Z, T* Y, cudaStream_t st);

template <typename T, typename V, int NB, int WARPS>
static eig_status tiled_launch_w(SpmmPlan* P, const T* X, T* Y, T* Z, size_t sm, cudaStream_t st) {
  TiledArgs a;
  a.n = P->n; a.R = P->R; a.C = P->C; a.cap = P->cap; a.rp_cap = (P->R + 1 + 7) / 8 * 8;
  a.chunk_ptr = P->chunk_ptr.as<int64_t>();
  a.chunks = P->chunks.as<TileChunk>();
  a.tcol = P->tcol.as<uint8_t>();
  a.tval = P->tval.p;
  a.trp = P->trp.as<uint16_t>();
  a.err = P->err.as<int>();
  auto kern = k_spmm_tiled<T, V, NB, WARPS>;
  EIG_CUDA_TRY(::eig::ensure_dyn_smem(kern, (int)sm));
  kern<<<(unsigned)P->nRB, WARPS * 32, sm, st>>>(a, X, Y, Z);
  EIG_LAUNCH_CHECK("k_spmm_tiled");
  return EIG_OK;
}

template <typename T, typename V, int NB>
eig_status tiled_launch(SpmmPlan* P, const T* X, T* Y, T* Z, cudaStream_t st) {
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // 8 warps when two CTAs fit on an SM, else fewer warps (fewer private transposed partials)
  if (tiled_smem<T, V, NB, 8>(P) <= (size_t)maxsm / 2) {
    EIG_TRY((tiled_launch_w<T, V, NB, 8>(P, X, Y, Z, tiled_smem<T, V, NB, 8>(P), st)));
  } else if (tiled_smem<T, V, NB, 4>(P) <= (size_t)maxsm) {
    EIG_TRY((tiled_launch_w<T, V, NB, 4>(P, X, Y, Z, tiled_smem<T, V, NB, 4>(P), st)));
  } else if (tiled_smem<T, V, NB, 2>(P) <= (size_t)maxsm) {
    EIG_TRY((tiled_launch_w<T, V, NB, 2>(P, X, Y, Z, tiled_smem<T, V, NB, 2>(P), st)));
  } else {
    return EIG_EUNSUPPORTED;
  }
  return transpose_reduce_launch<T, NB>(P, Z, Y, st);
}

#define EIG_TILED_INST(T, V)                                                                          \
  template eig_status tiled_launch<T, V, 1>(SpmmPlan*, const T*, T*, T*, cudaStream_t);               \
  template eig_status tiled_launch<T, V, 2>(SpmmPlan*, const T*, T*, T*, cudaStream_t);               \
  template eig_status tiled_launch<T, V, 4>(SpmmPlan*, const T*, T*, T*, cudaStream_t);               \
  template eig_status tiled_launch<T, V, 8>(SpmmPlan*, const T*, T*, T*, cudaStream_t);               \
  template eig_status tiled_launch<T, V, 16>(SpmmPlan*, const T*, T*, T*, cudaStream_t);              \
  template eig_status tiled_launch<T, V, 32>(SpmmPlan*, const T*, T*, T*, cudaStream_t);
EIG_TILED_INST(float, float)
EIG_TILED_INST(float, uint16_t)
EIG_TILED_INST(double, double)
EIG_TILED_INST(double, float)
EIG_TILED_INST(double, uint16_t)

}  // namespace eig
