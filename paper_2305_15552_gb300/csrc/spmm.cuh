// Symmetric half-stored SpMM plan (internal interface shared by the C ABI and the solvers).
#pragma once
#include "common.cuh"

namespace eig {

// One chunk of a tile (row block I, column block J): rows [ra, rb) of the row block, entries
// [ent_off, ent_off + nent) of the tiled arrays (nent_pad = nent rounded up to 16), row offsets
// trp[rp_off .. rp_off + rb - ra] relative to ent_off.
struct TileChunk {
  int64_t ent_off;
  int32_t nent_pad;
  int32_t J;
  int32_t rp_off;
  int16_t ra, rb;
  int32_t slot;    // scratch slot of the tile's transposed part, -1 for a tile inside the row block
  int32_t flags;   // bit 0: first chunk of its tile, bit 1: last chunk of its tile
};
static_assert(sizeof(TileChunk) == 32, "TileChunk layout");

struct SpmmPlan {
  int64_t n = 0, nnz = 0;
  int R = 256, C = 64;                  // row block / column block sizes
  int layout = EIG_LAYOUT_CSR;          // layout the kernels run on (eig_layout)
  int64_t nRB = 0, nCB = 0;
  eig_dtype val_type = EIG_F32;
  // matrix (owned when copied)
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  DevBuf own_rowptr, own_col, own_val;
  // tile lists: tiles of row block I are tile_col[tile_ptr[I] .. tile_ptr[I+1]), ascending J
  int64_t n_tiles = 0, n_slots = 0;
  DevBuf tile_ptr;     // int64[nRB+1]
  DevBuf tile_col;     // int32[n_tiles]
  DevBuf tile_slot;    // int32[n_tiles]: scratch slot of a non-local tile, -1 for local
  // transpose schedule: slots landing in column block J, ascending source row block
  DevBuf sched_ptr;    // int64[n_sched+1]
  DevBuf sched_cb;     // int32[n_sched]: column blocks that receive at least one slot
  DevBuf sched_slot;   // int32[n_slots]
  int64_t n_sched = 0;
  DevBuf diag;         // float64[n]: H_ii (used by the Jacobi preconditioner)
  // tile-contiguous copy of H (built by default): chunks of whole tile rows, each chunk's entries
  // contiguous (uint8 column within the tile + value), 16-byte aligned for bulk copies
  bool tiled = false;
  int cap = 0;                 // entries per chunk at most (multiple of 16)
  int64_t n_chunks = 0, tiled_entries = 0, tiled_rp = 0;
  DevBuf chunk_ptr;            // int64[nRB+1]
  DevBuf chunks;               // TileChunk[n_chunks]
  DevBuf tcol;                 // uint8[tiled_entries]
  DevBuf tval;                 // value type [tiled_entries]
  DevBuf trp;                  // uint16 row offsets within chunks
  DevBuf err;                  // int: device-side error flags (bounded waits that gave up)
  DevBuf scratch;      // transposed partial products, n_slots * C * nb * sizeof(T)
  // mirrored copy of H (both triangles; gather-only kernel): per row block of 256 rows, its
  // column tiles (64 columns) cut into panels of at most 24 tiles; per panel the rows ranked by
  // entry count, lane l of warp w taking the row of rank 32 w + l; per (panel, warp) a stream
  // of blocks of 32 lanes x 8 steps of (uint16 panel-local column, value), padded with
  // zero-valued entries on zero rows
  bool mirrored = false;
  int64_t m_npan = 0, m_nblk = 0, m_full_nnz = 0;
  DevBuf m_rbp;                      // int32[nRB+1]: panels of row block I
  DevBuf m_pt0, m_pnt;               // int32[m_npan]: first tile (into m_tcol) and tile count
  DevBuf m_tcol;                     // int32: column block of each tile of the mirrored matrix
  DevBuf m_perm;                     // uint8[m_npan * 256]: row (in its row block) of each slot
  DevBuf m_steps;                    // int32[m_npan * 8]: steps of each (panel, warp)
  DevBuf m_sboff;                    // int64[m_npan * 8 + 1]: first block of each (panel, warp)
  DevBuf m_bcol;                     // uint16[m_nblk * 256]
  DevBuf m_bval;                     // value type [m_nblk * 256]
  double algorithmic_bytes(int nb, size_t vec_bytes) const;
};

eig_status spmm_plan_build(SpmmPlan* P, const eig_csr_upper* H, int R, int C, int layout, int copy,
                           cudaStream_t st);
// Per row block of R rows, the ascending column blocks (of C) in which a sorted CSR has entries.
eig_status build_tile_lists(int64_t n, int R, int C, const int64_t* rowptr, const int32_t* col, cudaStream_t st,
                            DevBuf& tile_ptr, DevBuf& tile_col, std::vector<int64_t>& h_ptr,
                            std::vector<int32_t>& h_col);
// Builds the mirrored layout from the plan's CSR and tile lists (R = 256, C = 64 only).
eig_status spmm_plan_build_mirror(SpmmPlan* P, const std::vector<int64_t>& h_tptr,
                                  const std::vector<int32_t>& h_tcol, cudaStream_t st);
// Device bytes the mirrored layout needs while it is built (estimate).
size_t mirror_bytes_estimate(const SpmmPlan* P);
// Builds the tile-contiguous copy (called by spmm_plan_build).
eig_status spmm_plan_build_tiled(SpmmPlan* P, int cap, cudaStream_t st);
eig_status spmm_run(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, cudaStream_t st);
// One product of a batched launch: Y = H X on plan P (cheb: the fused Chebyshev step
// Y = alpha (H X - c X) - Qp, first = no Qp, X kept on inactive columns).
struct SpmmJob {
  SpmmPlan* P;
  const void* X;
  void* Y;
  const void* Qp;
  const int* active;
  double alpha, c;
  int first;
};
// Products of one shape -- block width nb, vector type vt, the plans' value type, plain or
// Chebyshev -- in one launch over their concatenated row blocks (the (instance, row block)
// work list of a batch); each product's sums are those of spmm_run / spmm_run_cheb.  Mirrored
// plans with FP32 values and nb 8 or 16 (FP32 or FP64 vectors); EIG_EUNSUPPORTED otherwise,
// with nothing launched.
eig_status spmm_run_batch(const SpmmJob* jobs, int count, int nb, eig_dtype vt, bool cheb, cudaStream_t st);
// Y(:, col) = H X(:, col) for blocks with row stride ld (one SpMV; mirrored layout only, else
// EIG_EUNSUPPORTED).
eig_status spmm_run_column(SpmmPlan* P, const void* X, void* Y, int ld, int col, eig_dtype vt, cudaStream_t st);
// Scratch bytes spmm_run needs for (nb, vec type); caller-provided scratch variant below.
size_t spmm_scratch_bytes(const SpmmPlan* P, int nb, eig_dtype vt);
eig_status spmm_run_with_scratch(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, void* scratch,
                                 cudaStream_t st);
// One Chebyshev step fused into the SpMM's epilogue (mirrored layout, nb 8 / 16 / 32; FP32 or
// FP64 vectors): Y = alpha (H X - c X) - Qp (no Qp when first), Y = X on columns with
// active[j] == 0 (device int[nb]).  EIG_EUNSUPPORTED for other layouts / shapes: the caller
// then runs the SpMM and the elementwise step separately.
eig_status spmm_run_cheb(SpmmPlan* P, const void* X, void* Y, int nb, eig_dtype vt, const void* Qp, const int* active,
                         double alpha, double c, int first, cudaStream_t st);

}  // namespace eig
